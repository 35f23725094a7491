// Point-target metrics (host launcher).
#pragma once

#include <cuda_runtime.h>

namespace bfp {

// Per-target output fields (doubles).
enum PtField : int {
  kPtPslrRange = 0, kPtPslrAz = 1, kPtIslrRange = 2, kPtIslrAz = 3, kPtWidthRange = 4, kPtWidthAz = 5,
  kPtPeak = 6, kPtSnr = 7, kPtNoise = 8, kPtPeakAz = 9, kPtPeakRg = 10, kPtReserved = 11,
  kPtMetricFields = 12
};
constexpr int kPtNoiseBlocks = 608;

size_t pt_workspace_bytes(long long n_az, long long n_rg);
cudaError_t launch_point_target_metrics(const void* img, bool img16, long long n_az, long long n_rg,
                                        const int* targets, int k, int guard, double* out, void* ws, cudaStream_t s);

}  // namespace bfp
