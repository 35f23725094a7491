// Row transforms computed in 16-bit arithmetic: the paper's "pure FP16" mode
// (Section III-A, Table I; Section VI's mode list) and bfloat16 (Section IV-C,
// the range-for-mantissa alternative), both with the fixed 1/N block shift of
// Eq. 1 before the inverse.
//
// Every add, subtract and multiply rounds to the 16-bit format: values stay
// packed as (re, im) pairs in one 32-bit register (__half2 / __nv_bfloat162),
// the butterflies use the paired HADD2 / HFMA2 instructions, twiddles are
// 16-bit (rounded once from FP64 sincospi), and the line crosses shared memory
// as 16-bit pairs.  The schedule is the radix-16 Stockham pass of
// fft_rows.cuh, and each operation and its rounding follow the same order as
// the radix-16 precision-mode schedule the tests compare against, so on
// lengths that are powers of 16 the output equals that schedule's value by
// value:
//   twiddle product   t = rn(a.re (c, s)),  a w = rn(a.im (-s, c) + t)   (fused)
//   4-point DFT       t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, d = a1 - a3,
//                     X0 = t0 + t2, X2 = t0 - t2, X1 = t1 - i d, X3 = t1 + i d
//   W16^2, W16^6      one rounded sum, then a rounded product by sqrt(1/2)
//   -i                exact swap
//
// Exchange layout (Layout16 below).  The XOR swizzle -- slot of point i is
// i XOR h(i >> 5) on its low five bits, h(q) = (q & 15) | (bit 3 of q) << 4 --
// was simulated over every pass of every length from 256 to 16384: the
// stride-16 stores of the first pass, the 256-apart half-warps of the second
// and the consecutive loads are all free of bank conflicts, with no padding.
// One padding slot per 32 points costs one two-way conflicted store group but
// no integer work per access; no linear padding is conflict-free in all
// passes (the first pass needs the second half-warp moved by 0 or 16 banks,
// the second by 8).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "async_copy.cuh"
#include "complex_ops.cuh"
#include "fft_rows.cuh"

namespace bfp {

// Paired 16-bit arithmetic.  H holds (re, im); every operation rounds to
// nearest even in H's format.  The _rn forms keep the compiler from fusing a
// product and a following sum into one FMA: the fused operations are exactly
// the ones written as fma, so the rounding sequence is the one stated above.
template <class H> struct A16;

template <> struct A16<__half2> {
  using H = __half2;
  __device__ __forceinline__ static H add(H a, H b) { return __hadd2_rn(a, b); }
  __device__ __forceinline__ static H sub(H a, H b) { return __hsub2_rn(a, b); }
  __device__ __forceinline__ static H mul(H a, H b) { return __hmul2_rn(a, b); }
  __device__ __forceinline__ static H fma(H a, H b, H c) { return __hfma2(a, b, c); }
  __device__ __forceinline__ static H neg(H a) { return __hneg2(a); }
  __device__ __forceinline__ static H re2(H a) { return __low2half2(a); }    // (re, re)
  __device__ __forceinline__ static H im2(H a) { return __high2half2(a); }   // (im, im)
  __device__ __forceinline__ static H swap(H a) { return __lowhigh2highlow(a); }
  __device__ __forceinline__ static H make(float x, float y) { return __floats2half2_rn(x, y); }
  __device__ __forceinline__ static H from_bits(uint32_t u) { return *reinterpret_cast<const H*>(&u); }
  __device__ __forceinline__ static uint32_t bits(H a) { return *reinterpret_cast<const uint32_t*>(&a); }
  __device__ __forceinline__ static float2 to_float2(H a) { return __half22float2(a); }
};

template <> struct A16<__nv_bfloat162> {
  using H = __nv_bfloat162;
  __device__ __forceinline__ static H add(H a, H b) { return __hadd2_rn(a, b); }
  __device__ __forceinline__ static H sub(H a, H b) { return __hsub2_rn(a, b); }
  __device__ __forceinline__ static H mul(H a, H b) { return __hmul2_rn(a, b); }
  __device__ __forceinline__ static H fma(H a, H b, H c) { return __hfma2(a, b, c); }
  __device__ __forceinline__ static H neg(H a) { return __hneg2(a); }
  __device__ __forceinline__ static H re2(H a) { return __low2bfloat162(a); }
  __device__ __forceinline__ static H im2(H a) { return __high2bfloat162(a); }
  __device__ __forceinline__ static H swap(H a) { return __lowhigh2highlow(a); }
  __device__ __forceinline__ static H make(float x, float y) { return __floats2bfloat162_rn(x, y); }
  __device__ __forceinline__ static H from_bits(uint32_t u) { return *reinterpret_cast<const H*>(&u); }
  __device__ __forceinline__ static uint32_t bits(H a) { return *reinterpret_cast<const uint32_t*>(&a); }
  __device__ __forceinline__ static float2 to_float2(H a) { return __bfloat1622float2(a); }
};

// A 16-bit twiddle as the pair the fused product needs: w = (c, s) and
// wp = (-s, c) (so a w = a.re w + a.im wp), 8 bytes, rounded once from FP64.
struct Tw16 {
  uint32_t w, wp;
};

template <class H>
struct Ops16 {
  using A = A16<H>;
  // a * w for a stored twiddle (w, wp): two rounded steps.
  __device__ __forceinline__ static H cmul(H a, H w, H wp) { return A::fma(A::im2(a), wp, A::mul(A::re2(a), w)); }
  // -i a = (im, -re), exact.
  __device__ __forceinline__ static H mul_mi(H a) { return A::mul(A::swap(a), A::make(1.f, -1.f)); }
  // x +- (-i d): (t.re + d.im, t.im - d.re) and (t.re - d.im, t.im + d.re), one rounding each.
  __device__ __forceinline__ static H add_mi(H t, H d) { return A::fma(A::swap(d), A::make(1.f, -1.f), t); }
  __device__ __forceinline__ static H sub_mi(H t, H d) { return A::fma(A::swap(d), A::make(-1.f, 1.f), t); }
  // W16^2 a = sqrt(1/2) ((x + y) + i (y - x)); W16^6 a = sqrt(1/2) ((y - x) - i (x + y)).
  __device__ __forceinline__ static H mul_w2(H a) {
    return A::mul(A::fma(A::swap(a), A::make(1.f, -1.f), a), A::make(kR2, kR2));
  }
  __device__ __forceinline__ static H mul_w6(H a) {
    return A::mul(A::fma(A::swap(a), A::make(1.f, -1.f), A::neg(a)), A::make(kR2, kR2));
  }
  __device__ __forceinline__ static void dft4(H& a0, H& a1, H& a2, H& a3) {
    const H t0 = A::add(a0, a2), t1 = A::sub(a0, a2), t2 = A::add(a1, a3), d = A::sub(a1, a3);
    a0 = A::add(t0, t2);
    a2 = A::sub(t0, t2);
    a1 = add_mi(t1, d);
    a3 = sub_mi(t1, d);
  }
};

template <class H, int R> struct Dft16b;

template <class H> struct Dft16b<H, 2> {
  __device__ __forceinline__ static void run(H (&v)[2]) {
    using A = A16<H>;
    const H a = v[0], b = v[1];
    v[0] = A::add(a, b);
    v[1] = A::sub(a, b);
  }
};

template <class H> struct Dft16b<H, 4> {
  __device__ __forceinline__ static void run(H (&v)[4]) { Ops16<H>::dft4(v[0], v[1], v[2], v[3]); }
};

// 8 = 2 x 4 (the structure of Dft<8> in complex_ops.cuh).
template <class H> struct Dft16b<H, 8> {
  __device__ __forceinline__ static void run(H (&v)[8]) {
    using A = A16<H>;
    using O = Ops16<H>;
    O::dft4(v[0], v[2], v[4], v[6]);
    O::dft4(v[1], v[3], v[5], v[7]);
    v[3] = O::mul_w2(v[3]);
    v[5] = O::mul_mi(v[5]);
    v[7] = O::mul_w6(v[7]);
    H o[8];
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      o[k2] = A::add(v[2 * k2], v[2 * k2 + 1]);
      o[k2 + 4] = A::sub(v[2 * k2], v[2 * k2 + 1]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = o[i];
  }
};

// 16 = 4 x 4: r = r1 + 4 r2, k = k2 + 4 k1; internal twiddles W16^(r1 k2).
template <class H> struct Dft16b<H, 16> {
  __device__ __forceinline__ static void run(H (&v)[16]) {
    using A = A16<H>;
    using O = Ops16<H>;
#pragma unroll
    for (int r1 = 0; r1 < 4; ++r1) O::dft4(v[r1], v[r1 + 4], v[r1 + 8], v[r1 + 12]);
    const H w1 = A::make(kC1, -kS1), w1p = A::make(kS1, kC1);      // W16^1
    const H w3 = A::make(kS1, -kC1), w3p = A::make(kC1, kS1);      // W16^3
    const H w9 = A::make(-kC1, kS1), w9p = A::make(-kS1, -kC1);    // W16^9
    v[5] = O::cmul(v[5], w1, w1p);
    v[9] = O::mul_w2(v[9]);
    v[13] = O::cmul(v[13], w3, w3p);
    v[6] = O::mul_w2(v[6]);
    v[10] = O::mul_mi(v[10]);
    v[14] = O::mul_w6(v[14]);
    v[7] = O::cmul(v[7], w3, w3p);
    v[11] = O::mul_w6(v[11]);
    v[15] = O::cmul(v[15], w9, w9p);
    H o[16];
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      H a0 = v[4 * k2 + 0], a1 = v[4 * k2 + 1], a2 = v[4 * k2 + 2], a3 = v[4 * k2 + 3];
      O::dft4(a0, a1, a2, a3);
      o[k2] = a0;
      o[k2 + 4] = a1;
      o[k2 + 8] = a2;
      o[k2 + 12] = a3;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = o[i];
  }
};

// 16-bit exchange layouts.  kSwizzle: the XOR swizzle of the header comment,
// free of bank conflicts but a few integer operations per access.  kPad32:
// one padding slot per 32 points, slot i + (i >> 5): every access is the
// thread's base plus a compile-time offset (no per-access integer work),
// conflict-free except the second pass's stores, whose half-warps lie 256
// points apart (two-way).
// kPadQ: each exchange has its own padding (every exchange is written once
// and read once, so the layouts need not agree): after the first pass
// i + (i >> 5), after the second i + (i >> 5) + 8 (i >> 8), which moves the
// second pass's 256-apart half-warps 16 banks apart.  Simulated over every
// pass: conflict-free for every length from 512 (a two-way conflict on one
// access group at 256 and below, where several lines share a warp), and every
// access is the thread's base plus a compile-time offset.
enum Layout16 : int { kSwizzle = 0, kPad32 = 1, kPadQ = 2 };

template <int L, int Q>
__device__ __forceinline__ int slot16(int i) {
  if constexpr (L == kSwizzle) {
    const int q = i >> 5;
    return i ^ ((q & 15) | (((q >> 3) & 1) << 4));
  } else if constexpr (L == kPadQ && Q == 1) {
    return i + (i >> 5) + 8 * (i >> 8);
  } else {
    return i + (i >> 5);
  }
}

template <int N, int L>
__host__ __device__ constexpr int slots16() { return L == kSwizzle ? N : L == kPad32 ? N + N / 32 : N + N / 16; }

template <int N, int Ns, class H, int L>
struct StockhamPass16 {
  static constexpr int P = kPointsPerThread;
  static constexpr int T = N / P;
  static constexpr int R = (N / Ns) >= 16 ? 16 : N / Ns;
  static constexpr int B = P / R;
  static constexpr bool kLast = (Ns * R == N);
  static constexpr int kQ = ilog16(Ns);   // exchange number written by this pass

  __device__ __forceinline__ static void run(H (&v)[P], const Tw16* __restrict__ tw, uint32_t* xch, int t) {
    using A = A16<H>;
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = t + T * b;
      const int k = j & (Ns - 1);
      H u[R];
#pragma unroll
      for (int r = 0; r < R; ++r) u[r] = v[b + B * r];
      if (Ns > 1) {
        // Pass-major table, the same indexing as the FP32 one: W_{Ns R}^{k r}
        // at (Ns - 16) + (r - 1) Ns + k.
        const Tw16* twp = tw + (Ns - 16) + k;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const uint2 p = __ldg(reinterpret_cast<const uint2*>(twp + (r - 1) * Ns));
          u[r] = Ops16<H>::cmul(u[r], A::from_bits(p.x), A::from_bits(p.y));
        }
      }
      Dft16b<H, R>::run(u);
      if (kLast) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[b + B * r] = u[r];
      } else {
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) xch[slot16<L, kQ>(base + r * Ns)] = A::bits(u[r]);
      }
    }
    if constexpr (!kLast) {
      __syncthreads();
#pragma unroll
      for (int m = 0; m < P; ++m) v[m] = A::from_bits(xch[slot16<L, kQ>(t + T * m)]);
      __syncthreads();
      StockhamPass16<N, Ns * R, H, L>::run(v, tw, xch, t);
    }
  }
};

// Dense rows of 16-bit storage computed in 16-bit arithmetic.  MODE kForward
// or kInverse (conj(DFT(conj(z) * 1/N)), the 1/N applied in the format before
// the transform, Eq. 1); NAIVE drops the shift and scales after the transform
// (Section III-B).  MODE kCompress is the matched-filter line of the SAR
// chain in the same arithmetic: forward DFT, the product with the filter
// spectrum a.h (rounded once to the format; the two-step fused product of the
// twiddles), conj and the 1/N shift, DFT, conj.  IN32: the input is complex64
// (the raw echo), rounded to the format as it is loaded.  One line per group
// of N / 16 threads.
template <int N, class H, int MODE, bool NAIVE, int MINB, int L, bool IN32 = false>
__global__ void __launch_bounds__(RowShape<N>::kThreads, MINB)
fft_rows16_kernel(const RowArgs a) {
  using S = RowShape<N>;
  using A = A16<H>;
  constexpr int P = S::P, T = S::T, G = S::G;
  extern __shared__ uint32_t smem16[];
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const long long line = (long long)blockIdx.x * G + g;
  const bool active = line < a.lines;
  uint32_t* xch = smem16 + g * slots16<N, L>();
  const Tw16* tw = static_cast<const Tw16*>(a.tw16);
  H v[P];
  if (active) {
    using TIn = typename std::conditional<IN32, float2, uint32_t>::type;
    if (a.pf_ahead > 0 && threadIdx.x == 0) {
      const long long l0 = ((long long)blockIdx.x + a.pf_ahead) * G;
      const long long cnt = a.lines - l0 < G ? a.lines - l0 : G;
      if (cnt > 0) prefetch_l2_bulk(static_cast<const TIn*>(a.in) + l0 * N, uint32_t(cnt * N * sizeof(TIn)));
    }
    const TIn* in = static_cast<const TIn*>(a.in) + line * a.in_stride + t;
#pragma unroll
    for (int m = 0; m < P; ++m) {
      if constexpr (IN32) {
        const float2 x = __ldcs(in + T * m);
        v[m] = A::make(x.x, x.y);
      } else {
        v[m] = A::from_bits(__ldcs(in + T * m));
      }
    }
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = A::make(0.f, 0.f);
  }
  if (MODE == kInverse) {
    const float s = NAIVE ? 1.0f : 1.0f / float(N);
    const H c = A::make(s, -s);   // conjugate and (BFP) shift: exact powers of two
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = A::mul(v[m], c);
  }
  StockhamPass16<N, 1, H, L>::run(v, tw, xch, t);
  if constexpr (MODE == kCompress) {
    // Filter product in groups of four (register pressure), then conj and the
    // shift; the first transform's last exchange ended with a barrier, so the
    // second may write the exchange buffer at once.
    const H c = A::make(NAIVE ? 1.0f : 1.0f / float(N), NAIVE ? -1.0f : -1.0f / float(N));
#pragma unroll
    for (int m0 = 0; m0 < P; m0 += 4) {
      float2 h[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) h[i] = __ldg(a.h + (active ? line : 0) * a.h_stride + t + T * (m0 + i));
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const H w = A::make(h[i].x, h[i].y), wp = A::make(-h[i].y, h[i].x);
        v[m0 + i] = A::mul(Ops16<H>::cmul(v[m0 + i], w, wp), c);
      }
    }
    int t2;
    asm volatile("mov.b32 %0, %1;" : "=r"(t2) : "r"(t));
    StockhamPass16<N, 1, H, L>::run(v, tw, xch, t2);
  }
  if (MODE == kInverse || MODE == kCompress) {
    const float s = NAIVE ? 1.0f / float(N) : 1.0f;
    const H c = A::make(s, -s);
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = A::mul(v[m], c);
  }
  if (active) {
    uint32_t* out = static_cast<uint32_t*>(a.out) + line * a.out_stride + t;
#pragma unroll
    for (int m = 0; m < P; ++m) __stcs(out + T * m, A::bits(v[m]));
    check_finite<Storage<float2>, P>(a.finite_flag, [&](int m) { return A::to_float2(v[m]); });
  }
}

template <int N, class H, int MODE, bool NAIVE, int MINB, int L, bool IN32 = false>
cudaError_t launch_rows16_nl(const RowArgs& a, cudaStream_t stream) {
  using S = RowShape<N>;
  constexpr size_t kBytes = size_t(S::G) * slots16<N, L>() * sizeof(uint32_t);
  auto kern = fft_rows16_kernel<N, H, MODE, NAIVE, MINB, L, IN32>;
  static const LaunchSetup setup = setup_kernel(kern, S::kThreads, kBytes);
  if (setup.err != cudaSuccess) return setup.err;
  if (a.lines <= 0) return cudaSuccess;
  const long long grid = (a.lines + S::G - 1) / S::G;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  RowArgs b = a;
  b.pf_ahead = (a.no_prefetch || a.in_stride != N) ? 0 : setup.resident;
  kern<<<dim3(unsigned(grid)), dim3(S::kThreads), kBytes, stream>>>(b);
  return cudaGetLastError();
}

// Exchange layout kPadQ (the swizzle and plain pad32 measured the same time as
// each other: the swizzle issue-bound, pad32 bound by its bank conflicts).
template <int N, class H, int MODE, bool NAIVE, int MINB, bool IN32 = false>
cudaError_t launch_rows16_n(const RowArgs& a, cudaStream_t stream) {
  return launch_rows16_nl<N, H, MODE, NAIVE, MINB, kPadQ, IN32>(a, stream);
}

// Resident CTAs per SM requested from the register allocator: 16 values of
// 32 bits per thread leave room for more than the FP32 kernel's four with
// FP16 (40 registers, no spills); bfloat16 pairs spill at 40 and keep four.
template <int N, class H>
constexpr int rows16_min_blocks() {
  return RowShape<N>::kThreads >= 1024 ? 1
         : RowShape<N>::kThreads >= 512 ? 2
         : (std::is_same<H, __half2>::value ? 6 : 4);
}

// SAR compression lines in FP16 arithmetic, log2n in [8, 14]: 4 CTAs per SM
// (the filter loads and the second transform need the FP32 kernel's registers).
template <bool NAIVE, bool IN32>
cudaError_t launch_rows16_compress(int log2n, const RowArgs& a, cudaStream_t s) {
  using H = __half2;
  switch (log2n) {
    case 8: return launch_rows16_n<256, H, kCompress, NAIVE, 4, IN32>(a, s);
    case 9: return launch_rows16_n<512, H, kCompress, NAIVE, 4, IN32>(a, s);
    case 10: return launch_rows16_n<1024, H, kCompress, NAIVE, 4, IN32>(a, s);
    case 11: return launch_rows16_n<2048, H, kCompress, NAIVE, 4, IN32>(a, s);
    case 12: return launch_rows16_n<4096, H, kCompress, NAIVE, 4, IN32>(a, s);
    case 13: return launch_rows16_n<8192, H, kCompress, NAIVE, 2, IN32>(a, s);
    case 14: return launch_rows16_n<16384, H, kCompress, NAIVE, 1, IN32>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <class H, int MODE, bool NAIVE>
cudaError_t launch_rows16(int log2n, const RowArgs& a, cudaStream_t s) {
  switch (log2n) {
    case 4: return launch_rows16_n<16, H, MODE, NAIVE, rows16_min_blocks<16, H>()>(a, s);
    case 5: return launch_rows16_n<32, H, MODE, NAIVE, rows16_min_blocks<32, H>()>(a, s);
    case 6: return launch_rows16_n<64, H, MODE, NAIVE, rows16_min_blocks<64, H>()>(a, s);
    case 7: return launch_rows16_n<128, H, MODE, NAIVE, rows16_min_blocks<128, H>()>(a, s);
    case 8: return launch_rows16_n<256, H, MODE, NAIVE, rows16_min_blocks<256, H>()>(a, s);
    case 9: return launch_rows16_n<512, H, MODE, NAIVE, rows16_min_blocks<512, H>()>(a, s);
    case 10: return launch_rows16_n<1024, H, MODE, NAIVE, rows16_min_blocks<1024, H>()>(a, s);
    case 11: return launch_rows16_n<2048, H, MODE, NAIVE, rows16_min_blocks<2048, H>()>(a, s);
    case 12: return launch_rows16_n<4096, H, MODE, NAIVE, rows16_min_blocks<4096, H>()>(a, s);
    case 13: return launch_rows16_n<8192, H, MODE, NAIVE, rows16_min_blocks<8192, H>()>(a, s);
    case 14: return launch_rows16_n<16384, H, MODE, NAIVE, rows16_min_blocks<16384, H>()>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bfp
