// FP64 metric reductions (host launchers).
#pragma once

#include <cuda_runtime.h>

namespace bfp {

constexpr int kMetricSums = 5;
constexpr int kMetricBlocks = 1024;            // upper bound on stage-1 blocks
constexpr size_t kMetricWorkspaceBytes = size_t(kMetricBlocks) * kMetricSums * sizeof(double);

// Blocks stage 1 uses for `count` points (1 .. kMetricBlocks).
int metric_blocks(long long count);

// Two-stage FP64 reduction of the five SQNR sums into out[5] (device).
// partials must hold metric_blocks(count) * kMetricSums doubles.
cudaError_t launch_sqnr_sums(const void* ref, bool ref16, const void* test, bool test16, long long count,
                             double* partials, double* out, cudaStream_t s);

// The same reduction with an explicit stage-1 block count (1 .. any); partials
// must hold blocks * kMetricSums doubles.
cudaError_t launch_sqnr_sums_blocks(const void* ref, bool ref16, const void* test, bool test16, long long count,
                                    double* partials, int blocks, double* out, cudaStream_t s);

}  // namespace bfp
