// Storage formats: load a complex point from HBM into FP32 registers and
// round it back on the way out.
//
//   float2   FP32 complex, 8 B / point
//   __half2  FP16 complex, 4 B / point (interleaved re, im; Section V's half2)
//   Fp8x2<>  FP8 complex, 2 B / point (OCP E4M3 or E5M2, Section VII)
//
// Conversions round to nearest even; FP8 conversions saturate to the largest
// finite value (satfinite).
#pragma once

#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cfloat>

namespace bfp {

struct E4M3 {};
struct E5M2 {};

template <class Fmt> struct alignas(2) Fp8x2 { __nv_fp8x2_storage_t bits; };

// The conversion intrinsics' name for each FP8 pair type.
template <class T> struct Fp8Format;
template <> struct Fp8Format<Fp8x2<E4M3>> { static constexpr __nv_fp8_interpretation_t kInterp = __NV_E4M3; };
template <> struct Fp8Format<Fp8x2<E5M2>> { static constexpr __nv_fp8_interpretation_t kInterp = __NV_E5M2; };

template <class T> struct Storage;

template <> struct Storage<float2> {
  static constexpr int kBytes = 8;
  __device__ __forceinline__ static float2 load(const float2* p) { return __ldcs(p); }
  __device__ __forceinline__ static void store(float2* p, float2 v) { __stcs(p, v); }
  __device__ __forceinline__ static float2 load_smem(const float2* p) { return *p; }
  // True when the stored value is finite (NaN fails both comparisons).
  __device__ __forceinline__ static bool finite(float2 v) { return fabsf(v.x) <= FLT_MAX && fabsf(v.y) <= FLT_MAX; }
};

template <> struct Storage<__half2> {
  static constexpr int kBytes = 4;
  __device__ __forceinline__ static float2 load(const __half2* p) {
    const unsigned int u = __ldcs(reinterpret_cast<const unsigned int*>(p));
    return __half22float2(*reinterpret_cast<const __half2*>(&u));
  }
  __device__ __forceinline__ static void store(__half2* p, float2 v) {
    const __half2 h = __float22half2_rn(v);
    __stcs(reinterpret_cast<unsigned int*>(p), *reinterpret_cast<const unsigned int*>(&h));
  }
  __device__ __forceinline__ static float2 load_smem(const __half2* p) { return __half22float2(*p); }
  // Round-to-nearest-even turns every magnitude >= 65520 into +-Inf.
  __device__ __forceinline__ static bool finite(float2 v) { return fabsf(v.x) < 65520.f && fabsf(v.y) < 65520.f; }
};

template <> struct Storage<Fp8x2<E4M3>> {
  static constexpr int kBytes = 2;
  __device__ __forceinline__ static float2 load(const Fp8x2<E4M3>* p) {
    const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2(p->bits, __NV_E4M3);
    return __half22float2(*reinterpret_cast<const __half2*>(&h));
  }
  __device__ __forceinline__ static void store(Fp8x2<E4M3>* p, float2 v) {
    p->bits = __nv_cvt_float2_to_fp8x2(v, __NV_SATFINITE, __NV_E4M3);
  }
  __device__ __forceinline__ static float2 load_smem(const Fp8x2<E4M3>* p) { return load(p); }
  // Satfinite stores turn +-Inf into the largest finite value; NaN stays NaN.
  __device__ __forceinline__ static bool finite(float2 v) { return v.x == v.x && v.y == v.y; }
};

template <> struct Storage<Fp8x2<E5M2>> {
  static constexpr int kBytes = 2;
  __device__ __forceinline__ static float2 load(const Fp8x2<E5M2>* p) {
    const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2(p->bits, __NV_E5M2);
    return __half22float2(*reinterpret_cast<const __half2*>(&h));
  }
  __device__ __forceinline__ static void store(Fp8x2<E5M2>* p, float2 v) {
    p->bits = __nv_cvt_float2_to_fp8x2(v, __NV_SATFINITE, __NV_E5M2);
  }
  __device__ __forceinline__ static float2 load_smem(const Fp8x2<E5M2>* p) { return load(p); }
  // Satfinite stores turn +-Inf into the largest finite value; NaN stays NaN.
  __device__ __forceinline__ static bool finite(float2 v) { return v.x == v.x && v.y == v.y; }
};

// Eight consecutive complex values (one 8-line segment of a corner-turned
// row) moved as 16-byte vectors: two for FP16, four for FP32.  The address
// must be 16-byte aligned.
template <class T> struct Seg8;
template <> struct Seg8<float2> {
  __device__ __forceinline__ static void load(const float2* p, float2 (&v)[8]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 q = __ldcs(reinterpret_cast<const float4*>(p) + i);
      v[2 * i] = make_float2(q.x, q.y);
      v[2 * i + 1] = make_float2(q.z, q.w);
    }
  }
  __device__ __forceinline__ static void store(float2* p, const float2 (&v)[8]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      __stcs(reinterpret_cast<float4*>(p) + i, make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y));
  }
};
// Raw FP16 segments: eight half2 words as two 16-byte vectors.
__device__ __forceinline__ void seg8_load_raw(const __half2* p, uint32_t (&w)[8]) {
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const uint4 q = __ldcs(reinterpret_cast<const uint4*>(p) + i);
    w[4 * i] = q.x;
    w[4 * i + 1] = q.y;
    w[4 * i + 2] = q.z;
    w[4 * i + 3] = q.w;
  }
}
__device__ __forceinline__ void seg8_store_raw(__half2* p, const uint32_t (&w)[8]) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
    __stcs(reinterpret_cast<uint4*>(p) + i, make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]));
}
__device__ __forceinline__ uint32_t half2_bits(float2 v) {
  const __half2 h = __float22half2_rn(v);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ float2 bits_half2(uint32_t u) { return __half22float2(*reinterpret_cast<const __half2*>(&u)); }

template <> struct Seg8<__half2> {
  __device__ __forceinline__ static void load(const __half2* p, float2 (&v)[8]) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const uint4 q = __ldcs(reinterpret_cast<const uint4*>(p) + i);
      const unsigned int w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) v[4 * i + j] = __half22float2(*reinterpret_cast<const __half2*>(&w[j]));
    }
  }
  __device__ __forceinline__ static void store(__half2* p, const float2 (&v)[8]) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      unsigned int w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const __half2 h = __float22half2_rn(v[4 * i + j]);
        w[j] = *reinterpret_cast<const unsigned int*>(&h);
      }
      __stcs(reinterpret_cast<uint4*>(p) + i, make_uint4(w[0], w[1], w[2], w[3]));
    }
  }
};

// Naive FP16 output of an unshifted inverse (Section III-B): the unnormalised
// result is stored to half first (overflowing to +-Inf beyond 65504) and only
// then multiplied by 1/N, in half.
__device__ __forceinline__ float2 naive_half_then_scale(float2 v, float inv_n) {
  const __half2 h = __float22half2_rn(v);
  const __half2 s = __hmul2(h, __float2half2_rn(inv_n));
  return __half22float2(s);
}

}  // namespace bfp
