// Rows computed in 16-bit arithmetic (fft_half.cuh): FP16 (the paper's pure
// FP16 mode) and bfloat16, forward and inverse, with or without the shift.
#include "fft_half.cuh"
#include "launch.h"

namespace bfp {

cudaError_t launch_rows16_f16(int log2n, int mode, bool naive, const RowArgs& a, cudaStream_t s) {
  if (mode == kForward) return launch_rows16<__half2, kForward, false>(log2n, a, s);
  if (mode != kInverse) return cudaErrorInvalidValue;
  return naive ? launch_rows16<__half2, kInverse, true>(log2n, a, s)
               : launch_rows16<__half2, kInverse, false>(log2n, a, s);
}

cudaError_t launch_rows16_compress_f16(int log2n, bool in32, bool naive, const RowArgs& a, cudaStream_t s) {
  if (in32) return naive ? launch_rows16_compress<true, true>(log2n, a, s) : launch_rows16_compress<false, true>(log2n, a, s);
  return naive ? launch_rows16_compress<true, false>(log2n, a, s) : launch_rows16_compress<false, false>(log2n, a, s);
}

cudaError_t launch_rows16_bf16(int log2n, int mode, const RowArgs& a, cudaStream_t s) {
  if (mode == kForward) return launch_rows16<__nv_bfloat162, kForward, false>(log2n, a, s);
  if (mode == kInverse) return launch_rows16<__nv_bfloat162, kInverse, false>(log2n, a, s);
  return cudaErrorInvalidValue;
}

// Pass-major 16-bit twiddle table of a length-n transform: entry
// (Ns - 16) + (r - 1) Ns + k holds w = W_{Ns R}^{k r} = (c, s) and
// wp = (-s, c), each part evaluated in FP64 (sincospi of an exact dyadic
// fraction) and rounded once to the 16-bit format.
template <class H>
__global__ void twiddle16_kernel(Tw16* tw, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 16) return;
  int ns = 16;
  while (ns * 16 < n && i >= ns * 16 - 16) ns *= 16;
  const int radix = (n / ns) >= 16 ? 16 : n / ns;
  const int local = i - (ns - 16);
  const int r = local / ns + 1;
  const int k = local - (r - 1) * ns;
  double s, c;
  sincospi(-2.0 * double(k * r) / double(ns * radix), &s, &c);
  H w, wp;
  if constexpr (std::is_same<H, __half2>::value) {
    w = __halves2half2(__double2half(c), __double2half(s));
    wp = __halves2half2(__double2half(-s), __double2half(c));
  } else {
    w = __halves2bfloat162(__double2bfloat16(c), __double2bfloat16(s));
    wp = __halves2bfloat162(__double2bfloat16(-s), __double2bfloat16(c));
  }
  tw[i] = Tw16{A16<H>::bits(w), A16<H>::bits(wp)};
}

cudaError_t launch_twiddles16(void* tw, int n, bool bf16) {
  const int threads = 256, blocks = (n + threads - 1) / threads;
  if (bf16) {
    twiddle16_kernel<__nv_bfloat162><<<blocks, threads>>>(static_cast<Tw16*>(tw), n);
  } else {
    twiddle16_kernel<__half2><<<blocks, threads>>>(static_cast<Tw16*>(tw), n);
  }
  return cudaGetLastError();
}

}  // namespace bfp
