// Uneven-batch persistent launch (host interface).
#pragma once

#include <cuda_runtime.h>

#include "fft_rows.cuh"

namespace bfp {

struct UnevenTask {
  int log2n;     // length class
  int first;     // first line of the task in the sorted line list
  int count;     // lines in the task (65536 / N, fewer for the last task of a class)
  int pad;
};

struct UnevenArgs {
  const void* in;
  void* out;
  const long long* line_off;     // point offset of every line, sorted by task
  const UnevenTask* tasks;
  int num_tasks;
  const float2* const* tw;       // per-length twiddle tables, indexed by log2 N
  const float2* const* tw4;      // per-length four-step tables (N >= 8192), indexed by log2 N
  int* counter;                  // task counter (reset before every launch)
  int* status;
  int prefetch;                  // nonzero: prefetch each CTA's lines of the next task into L2
  int* finite_flag;              // non-null: record non-finite outputs here (BFPFFT_CHECK_FINITE)
  int fs_h16;                    // FP16 storage: four-step lines exchange their rows as FP16 words
};

// Row and output buffers of the longest four-step line (N1 = 16), for the
// storage type TS.
template <class TS>
constexpr size_t uneven_smem_bytes() { return fourstep_smem_bytes<TS, 16>(); }
constexpr int kUnevenTaskPoints = 65536;

// Storage kind: 0 FP32, 1 FP16 (block-floating-point), 2 E4M3, 3 E5M2.
cudaError_t uneven_max_clusters(int kind, bool inverse, int* max_clusters);
cudaError_t launch_uneven(int kind, bool inverse, const UnevenArgs& a, int clusters, cudaStream_t s);

}  // namespace bfp
