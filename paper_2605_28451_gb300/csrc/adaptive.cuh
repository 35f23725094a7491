// Adaptive per-line block exponents (Section VIII, Limitations: a block-max
// reduction that picks the exponent per block, the alternative the paper
// names to its fixed 1/N shift for inputs of arbitrary amplitude).
//
// A block is one transform line.  After the line's transform(s) in FP32
// registers, the CTA reduces the largest |Re| or |Im| of the line, m, and
// takes its exponent e as the smallest integer with m 2^-e <= 2^14, read
// straight from the bits of the FP32 maximum (no logarithm, no rounding).
// The line is stored as FP16 mantissas round(v 2^-e) -- the largest
// component lands in (2^13, 2^14], a factor of four below FP16's 65504 --
// plus one int32 exponent; its value is mantissa * 2^e.  On input, a line's
// exponent scales its FP16 mantissas back to values (exactly: powers of two)
// before the transform, so a chain of adaptive transforms never overflows
// and never loses the line's power-of-two scale.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "fft_rows.cuh"

namespace bfp {

constexpr int kAdaptiveLimitLog2 = 14;   // stored block maximum <= 2^14

// 2^k as FP32 for k in [-126, 127] (a normal power of two, built from its bits).
__device__ __forceinline__ float exp2i(int k) { return __int_as_float((k + 127) << 23); }

// v * 2^k, exact whenever the result is a normal FP32 number; |k| <= 252.  The
// two factors have the sign of k, so no intermediate overflows or underflows
// before the result does.
__device__ __forceinline__ float2 scale_pow2(float2 v, int k) {
  const int h = k / 2;
  const float fa = exp2i(h), fb = exp2i(k - h);
  return make_float2(v.x * fa * fb, v.y * fa * fb);
}

// Smallest e with m 2^-e <= 2^14 for the FP32 value m whose bit pattern is
// `bits` (positive, finite, nonzero): m = 1.f 2^E, so e = E - 14 when m is a
// power of two (f = 0) and E - 13 otherwise.  Subnormal m = bits 2^-149.
__device__ __forceinline__ int block_exponent_of(uint32_t bits) {
  int E;
  bool pow2;
  if (bits >= 0x00800000u) {
    E = int(bits >> 23) - 127;
    pow2 = (bits & 0x007fffffu) == 0u;
  } else {
    E = (31 - __clz(int(bits))) - 149;
    pow2 = (bits & (bits - 1u)) == 0u;
  }
  return pow2 ? E - kAdaptiveLimitLog2 : E - kAdaptiveLimitLog2 + 1;
}

// Rows with adaptive exponents: FP16 mantissas out (half2) plus out_exp[line];
// input TIn = __half2 mantissas with optional in_exp[line], or float2 values.
// MODE: forward, inverse (the normalised inverse, with its 1/N folded into the
// pre-inverse conjugate as in Eq. 1) or compress (forward, filter, inverse).
template <int N, class TIn, int MODE>
__global__ void __launch_bounds__(RowShape<N>::kThreads, RowShape<N>::kMinBlocksDense)
fft_rows_adaptive_kernel(const RowArgs a) {
  using S = RowShape<N>;
  constexpr int P = S::P, T = S::T, G = S::G;
  extern __shared__ float2 smem_ad[];
  __shared__ uint32_t warp_max[32];
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const long long line = (long long)blockIdx.x * G + g;
  const bool active = line < a.lines;
  float2* sm = smem_ad + g * S::kSmemPerLine;
  float2 v[P];
  if (active) {
    if (a.pf_ahead > 0 && threadIdx.x == 0) {
      const long long l0 = ((long long)blockIdx.x + a.pf_ahead) * G;
      const long long cnt = a.lines - l0 < G ? a.lines - l0 : G;
      if (cnt > 0) prefetch_l2_bulk(static_cast<const TIn*>(a.in) + l0 * N, uint32_t(cnt * N * sizeof(TIn)));
    }
    const TIn* in = static_cast<const TIn*>(a.in) + line * a.in_stride + t;
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = Storage<TIn>::load(in + T * m);
    if (a.in_exp != nullptr) {
      const int ei = max(-252, min(252, a.in_exp[line]));
#pragma unroll
      for (int m = 0; m < P; ++m) v[m] = scale_pow2(v[m], ei);
    }
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = make_float2(0.f, 0.f);
  }
  row_compute<N, MODE, false, false>(v, a, sm, t, line);

  // Block maximum of |Re|, |Im| over the line.  Non-negative floats order like
  // their bit patterns, so the reduction runs on unsigned integers.
  uint32_t mx = 0u;
#pragma unroll
  for (int m = 0; m < P; ++m)
    mx = max(mx, max(__float_as_uint(fabsf(v[m].x)), __float_as_uint(fabsf(v[m].y))));
  if constexpr (T < 32) {
    // a line is T consecutive lanes of one warp (T a power of two)
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  } else {
    constexpr int W = T / 32;   // warps per line
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = mx;
    __syncthreads();
    if constexpr (W > 1) {
      mx = 0u;
#pragma unroll
      for (int w = 0; w < W; ++w) mx = max(mx, warp_max[g * W + w]);
    }
  }
  // Zero lines keep e = 0; a line holding Inf or NaN is stored unscaled.
  const int e = (mx != 0u && mx < 0x7f800000u) ? block_exponent_of(mx) : 0;
  if (active) {
    __half2* out = static_cast<__half2*>(a.out) + line * a.out_stride + t;
#pragma unroll
    for (int m = 0; m < P; ++m) Storage<__half2>::store(out + T * m, scale_pow2(v[m], -e));
    if (t == 0) a.out_exp[line] = e;
    check_finite<Storage<__half2>, P>(a.finite_flag, [&](int m) { return scale_pow2(v[m], -e); });
  }
}

template <int N, class TIn, int MODE>
cudaError_t launch_adaptive_n(const RowArgs& a, cudaStream_t stream) {
  using S = RowShape<N>;
  auto kern = fft_rows_adaptive_kernel<N, TIn, MODE>;
  static const LaunchSetup setup = setup_kernel(kern, S::kThreads, S::kSmemBytes);
  if (setup.err != cudaSuccess) return setup.err;
  if (a.lines <= 0) return cudaSuccess;
  const long long grid = (a.lines + S::G - 1) / S::G;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  RowArgs b = a;
  // Dense rows in device memory: each CTA prefetches the lines of the CTA one
  // resident wave later into L2 (as the default row variant does).
  b.pf_ahead = (a.no_prefetch || a.in_stride != N) ? 0 : setup.resident;
  kern<<<dim3(unsigned(grid)), dim3(S::kThreads), S::kSmemBytes, stream>>>(b);
  return cudaGetLastError();
}

// Dispatch on log2 N in [4, 14] (lines held by one CTA).
template <class TIn, int MODE>
cudaError_t launch_rows_adaptive(int log2n, const RowArgs& a, cudaStream_t s) {
  switch (log2n) {
    case 4: return launch_adaptive_n<16, TIn, MODE>(a, s);
    case 5: return launch_adaptive_n<32, TIn, MODE>(a, s);
    case 6: return launch_adaptive_n<64, TIn, MODE>(a, s);
    case 7: return launch_adaptive_n<128, TIn, MODE>(a, s);
    case 8: return launch_adaptive_n<256, TIn, MODE>(a, s);
    case 9: return launch_adaptive_n<512, TIn, MODE>(a, s);
    case 10: return launch_adaptive_n<1024, TIn, MODE>(a, s);
    case 11: return launch_adaptive_n<2048, TIn, MODE>(a, s);
    case 12: return launch_adaptive_n<4096, TIn, MODE>(a, s);
    case 13: return launch_adaptive_n<8192, TIn, MODE>(a, s);
    case 14: return launch_adaptive_n<16384, TIn, MODE>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bfp
