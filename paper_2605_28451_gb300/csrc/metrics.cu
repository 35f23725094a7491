// FP64 reductions for the quality metrics (Section IV-B's scale-aligned SQNR).
//
// For a reference r and a test t of `count` complex points each (float2 or
// __half2 storage), the five sums
//
//   s0 = sum |r|^2        s1 = sum |t|^2        s2 = Re sum conj(t) r
//   s3 = sum |r - t|^2    s4 = number of non-finite test points
//
// give the aligned SQNR 10 log10(s0 / (s0 - s2^2 / s1)) (optimal real scale
// alpha = s2 / s1) and the unaligned one 10 log10(s0 / s3).  Stage 1: a grid
// of kMetricBlocks blocks accumulates FP64 partials into a workspace; stage 2:
// one block adds the partials in a fixed order, so the result is bitwise
// reproducible run to run.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "metrics.h"

namespace bfp {

namespace {

constexpr int kThreads = 256;

template <class T> __device__ __forceinline__ double2 load_c(const T* p, long long i);
template <> __device__ __forceinline__ double2 load_c<float2>(const float2* p, long long i) {
  const float2 v = p[i];
  return make_double2(v.x, v.y);
}
template <> __device__ __forceinline__ double2 load_c<__half2>(const __half2* p, long long i) {
  const float2 v = __half22float2(p[i]);
  return make_double2(v.x, v.y);
}

__device__ __forceinline__ void block_sum5(double (&v)[kMetricSums], double* out) {
  __shared__ double red[kMetricSums][kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kMetricSums; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[k][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < kMetricSums) {
    double x = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) x += red[threadIdx.x][w];
    out[threadIdx.x] = x;
  }
}

template <class TR, class TT>
__global__ void __launch_bounds__(kThreads) sqnr_partials_kernel(const TR* __restrict__ ref,
                                                                 const TT* __restrict__ test, long long count,
                                                                 double* __restrict__ partials) {
  double acc[kMetricSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < count;
       i += (long long)gridDim.x * kThreads) {
    const double2 r = load_c(ref, i);
    const double2 t = load_c(test, i);
    if (!isfinite(t.x) || !isfinite(t.y)) {
      acc[4] += 1.0;
      continue;
    }
    const double dx = r.x - t.x, dy = r.y - t.y;
    acc[0] += r.x * r.x + r.y * r.y;
    acc[1] += t.x * t.x + t.y * t.y;
    acc[2] += t.x * r.x + t.y * r.y;
    acc[3] += dx * dx + dy * dy;
  }
  block_sum5(acc, partials + (long long)blockIdx.x * kMetricSums);
}

__global__ void __launch_bounds__(kThreads) sqnr_final_kernel(const double* __restrict__ partials, int blocks,
                                                              double* __restrict__ out) {
  double acc[kMetricSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < blocks; b += kThreads) {
#pragma unroll
    for (int k = 0; k < kMetricSums; ++k) acc[k] += partials[(long long)b * kMetricSums + k];
  }
  block_sum5(acc, out);
}

template <class TR, class TT>
cudaError_t launch_typed(const void* ref, const void* test, long long count, double* partials, int blocks,
                         double* out, cudaStream_t s) {
  sqnr_partials_kernel<TR, TT><<<blocks, kThreads, 0, s>>>(static_cast<const TR*>(ref),
                                                           static_cast<const TT*>(test), count, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sqnr_final_kernel<<<1, kThreads, 0, s>>>(partials, blocks, out);
  return cudaGetLastError();
}

}  // namespace

int metric_blocks(long long count) {
  long long b = (count + kThreads * 16 - 1) / (kThreads * 16);
  if (b < 1) b = 1;
  if (b > kMetricBlocks) b = kMetricBlocks;
  return int(b);
}

cudaError_t launch_sqnr_sums_blocks(const void* ref, bool ref16, const void* test, bool test16, long long count,
                                    double* partials, int blocks, double* out, cudaStream_t s) {
  if (ref16) {
    if (test16) return launch_typed<__half2, __half2>(ref, test, count, partials, blocks, out, s);
    return launch_typed<__half2, float2>(ref, test, count, partials, blocks, out, s);
  }
  if (test16) return launch_typed<float2, __half2>(ref, test, count, partials, blocks, out, s);
  return launch_typed<float2, float2>(ref, test, count, partials, blocks, out, s);
}

cudaError_t launch_sqnr_sums(const void* ref, bool ref16, const void* test, bool test16, long long count,
                             double* partials, double* out, cudaStream_t s) {
  const int blocks = metric_blocks(count);
  if (ref16) {
    if (test16) return launch_typed<__half2, __half2>(ref, test, count, partials, blocks, out, s);
    return launch_typed<__half2, float2>(ref, test, count, partials, blocks, out, s);
  }
  if (test16) return launch_typed<float2, __half2>(ref, test, count, partials, blocks, out, s);
  return launch_typed<float2, float2>(ref, test, count, partials, blocks, out, s);
}

}  // namespace bfp
