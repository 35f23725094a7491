// Complex arithmetic and small DFT blocks for the register-resident butterflies.
//
// All arithmetic is FP32 (float2 = re, im), whatever the storage type: the
// paper's FP16-storage / FP32-compute mode (Section VI), which keeps every
// multiply-add of a butterfly in FP32 registers and rounds to FP16 only where
// data leaves the chip.
//
// The blocks compute the forward DFT  X[k] = sum_r v[r] exp(-2 pi i r k / R)
// for R = 2, 4, 8, 16, in natural output order.  The inverse is never needed:
// the inverse transform is realised as conj(FFT(conj z)) (Section III-B).
#pragma once

#include <cuda_runtime.h>

namespace bfp {

// Packed FP32 (sm_100-family f32x2): one instruction adds or subtracts both
// components of a complex value held as a 64-bit register pair.
#ifndef BFP_F32X2
#define BFP_F32X2 1
#endif

__device__ __forceinline__ unsigned long long as_u64(float2 a) { return *reinterpret_cast<unsigned long long*>(&a); }
__device__ __forceinline__ float2 as_f2(unsigned long long u) { return *reinterpret_cast<float2*>(&u); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
#if BFP_F32X2
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(as_u64(a)), "l"(as_u64(b)));
  return as_f2(r);
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
#if BFP_F32X2
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(as_u64(a)), "l"(as_u64(b)));
  return as_f2(r);
#else
  return make_float2(a.x - b.x, a.y - b.y);
#endif
}
// Both components times the same real factor.
__device__ __forceinline__ float2 cmul_real2(float2 a, float s) {
#if BFP_F32X2
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(as_u64(a)), "l"(as_u64(make_float2(s, s))));
  return as_f2(r);
#else
  return make_float2(a.x * s, a.y * s);
#endif
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i
__device__ __forceinline__ float2 cmul_mi(float2 a) { return make_float2(a.y, -a.x); }

// Constant twiddles of the 16-point block, W16^e = exp(-2 pi i e / 16).
constexpr float kC1 = 0.92387953251128675613f;   // cos(pi/8)
constexpr float kS1 = 0.38268343236508977173f;   // sin(pi/8)
constexpr float kR2 = 0.70710678118654752440f;   // sqrt(1/2)

// (x + iy) * W16^2 = sqrt(1/2) * ((x + y) + i (y - x))
__device__ __forceinline__ float2 mul_w16_2(float2 a) { return cmul_real2(make_float2(a.x + a.y, a.y - a.x), kR2); }
// (x + iy) * W16^6 = sqrt(1/2) * ((y - x) - i (x + y))
__device__ __forceinline__ float2 mul_w16_6(float2 a) { return cmul_real2(make_float2(a.y - a.x, -a.x - a.y), kR2); }
__device__ __forceinline__ float2 mul_w16_1(float2 a) { return cmul(a, make_float2(kC1, -kS1)); }
__device__ __forceinline__ float2 mul_w16_3(float2 a) { return cmul(a, make_float2(kS1, -kC1)); }
__device__ __forceinline__ float2 mul_w16_9(float2 a) { return cmul(a, make_float2(-kC1, kS1)); }

// 4-point forward DFT in place: (a0, a1, a2, a3) -> (X0, X1, X2, X3).
// e = -i (a1 - a3) is formed with two scalar subtractions straight into the
// swapped order, so every other step is one packed add or subtract.
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
  const float2 t2 = cadd(a1, a3);
  const float2 e = make_float2(a1.y - a3.y, a3.x - a1.x);
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, e);
  a3 = csub(t1, e);
}

template <int R> struct Dft;

template <> struct Dft<2> {
  __device__ __forceinline__ static void run(float2 (&v)[2]) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <> struct Dft<4> {
  __device__ __forceinline__ static void run(float2 (&v)[4]) { dft4(v[0], v[1], v[2], v[3]); }
};

// 8 = 2 x 4: r = r1 + 2 r2, k = k2 + 4 k1.
template <> struct Dft<8> {
  __device__ __forceinline__ static void run(float2 (&v)[8]) {
    dft4(v[0], v[2], v[4], v[6]);           // r1 = 0 -> a0[k2] at v[0,2,4,6]
    dft4(v[1], v[3], v[5], v[7]);           // r1 = 1 -> a1[k2] at v[1,3,5,7]
    // a1[k2] *= W8^k2
    v[3] = mul_w16_2(v[3]);
    v[5] = cmul_mi(v[5]);
    v[7] = mul_w16_6(v[7]);
    float2 o[8];
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      o[k2] = cadd(v[2 * k2], v[2 * k2 + 1]);
      o[k2 + 4] = csub(v[2 * k2], v[2 * k2 + 1]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = o[i];
  }
};

// 16 = 4 x 4: r = r1 + 4 r2, k = k2 + 4 k1.
template <> struct Dft<16> {
  __device__ __forceinline__ static void run(float2 (&v)[16]) {
#pragma unroll
    for (int r1 = 0; r1 < 4; ++r1) dft4(v[r1], v[r1 + 4], v[r1 + 8], v[r1 + 12]);
    // a[r1][k2] sits at v[r1 + 4 k2]; multiply by W16^(r1 k2).
    v[5] = mul_w16_1(v[5]);
    v[9] = mul_w16_2(v[9]);
    v[13] = mul_w16_3(v[13]);
    v[6] = mul_w16_2(v[6]);
    v[10] = cmul_mi(v[10]);
    v[14] = mul_w16_6(v[14]);
    v[7] = mul_w16_3(v[7]);
    v[11] = mul_w16_6(v[11]);
    v[15] = mul_w16_9(v[15]);
    // DFT-4 over r1 for each k2; X[k2 + 4 k1] = result k1.
    float2 o[16];
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      float2 a0 = v[4 * k2 + 0], a1 = v[4 * k2 + 1], a2 = v[4 * k2 + 2], a3 = v[4 * k2 + 3];
      dft4(a0, a1, a2, a3);
      o[k2] = a0;
      o[k2 + 4] = a1;
      o[k2 + 8] = a2;
      o[k2 + 12] = a3;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = o[i];
  }
};

}  // namespace bfp
