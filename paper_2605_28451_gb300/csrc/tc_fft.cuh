// Radix-16 passes on the 5th-generation tensor cores (tcgen05) for N = 4096.
//
// A radix-16 pass over 256 butterflies is a dense real contraction:
//
//   D[j][n] = sum_k A[j][k] B[n][k],   j < 256 butterflies, n, k < 32
//
// where row j of A holds the 16 (twiddled) complex inputs of butterfly j as
// interleaved (re, im) FP16 pairs (k = 2 r + c), and B is the 16-point DFT
// matrix W16^{qr} = exp(-2 pi i q r / 16) in real form: B[2q][2r] = Re W,
// B[2q][2r+1] = -Im W, B[2q+1][2r] = Im W, B[2q+1][2r+1] = Re W.  Row j of D
// (FP32, in tensor memory) is then the 16 complex outputs of butterfly j.
//
// Per pass: one thread issues four tcgen05.mma (two M = 128 tiles x two
// K = 16 steps, N = 32) from shared-memory descriptors (K-major, no swizzle,
// 8 x 16-byte core matrices), commits them to an mbarrier, and every thread
// reads its D row back with tcgen05.ld.  The producer side applies the next
// pass's Stockham twiddle in FP32 and stores the FP16 result straight into
// the next pass's A tile (the A tile is the inter-pass exchange), so each
// pass moves 4 B per point into shared memory and the tensor core reads it
// back once.  FP16 operands, FP32 accumulation: every pass boundary is an FP16
// storage point, so the inverse relies on the 1/N shift (Eq. 1) like the
// paper's half2 kernel.
//
// Rows: butterfly j of pass p sits in A/D row rho_p(j); thread tau < 128
// (TMEM lane tau) handles the butterflies in rows tau and 128 + tau, one per
// M tile.  rho_p keep every shared-memory store of the producer free of bank
// conflicts (below).  Eight 128-thread CTAs share an SM, so that while one
// waits for its MMAs the others load, twiddle and store.
//
// Waits are bounded; on expiry the CTA records a timeout, waits (bounded) for
// its last commit, frees its tensor memory and returns.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "fft_rows.cuh"

namespace bfp {

namespace tc {

constexpr int kN = 4096;
constexpr int kB = 256;              // butterflies per pass
constexpr int kThreads = 128;        // one per TMEM lane; each owns the lane in both M tiles
constexpr int kLbo = 128;            // bytes between K-adjacent core matrices
constexpr int kSbo = 512;            // bytes between 8-row groups (4 core matrices of K = 32)
constexpr int kABytes = kB * 64;     // 256 rows x 32 FP16
constexpr int kBBytes = 32 * 64;     // 32 rows x 32 FP16
constexpr int kLineBytes = kN * 4;   // one FP16 line
constexpr uint32_t kTmemCols = 64;   // two 128 x 32 FP32 accumulators
constexpr int kCtasPerSm = 8;        // 64 registers, 64 TMEM columns, 26 KB of shared memory each
constexpr int kTwPitch = 18;         // twiddle rows in shared memory: 18 entries (144 B) apart
constexpr int kTwBytes = 2 * 16 * kTwPitch * 8;
// Shared memory: A | 3 B matrices | twiddle rows | mbarrier | TMEM slot.
constexpr int kBOff = kABytes;
constexpr int kTwOff = kBOff + 3 * kBBytes;
constexpr int kBarOff = (kTwOff + kTwBytes + 15) / 16 * 16;
constexpr int kSmemBytes = kBarOff + 16;

// K-major canonical layout without swizzle: byte offset of element (row, k).
__host__ __device__ constexpr int kmaj(int row, int k) {
  return (row / 8) * kSbo + (k / 8) * kLbo + (row % 8) * 16 + (k % 8) * 2;
}

// Row of butterfly j in pass P (0, 1, 2) and its inverse.  The bank of a
// 4-byte store into the A tile is (row % 8) * 4 + (k-pair % 4), so the maps
// are chosen (GF(2)-linear in the 8 bits of j) such that the 32 lanes of a
// warp always hit 32 different banks:
//   P = 0: row bits = j bits (0, 1, 2, 4, 5, 3, 6, 7)
//   P = 1: row bits = (j4, j5, j6 ^ j0, j1, j2, j3, j6, j7)
//   P = 2: identity (the last pass stores X[j + 256 q] coalesced)
// The pass-0 inputs go in as 16-byte stores, four k-pairs of one row each.
__device__ __forceinline__ int bit(int x, int b) { return (x >> b) & 1; }

template <int P>
__device__ __forceinline__ int row_of(int j) {
  if constexpr (P == 0) {
    return bit(j, 0) | bit(j, 1) << 1 | bit(j, 2) << 2 | bit(j, 4) << 3 | bit(j, 5) << 4 | bit(j, 3) << 5 |
           bit(j, 6) << 6 | bit(j, 7) << 7;
  } else if constexpr (P == 1) {
    return bit(j, 4) | bit(j, 5) << 1 | (bit(j, 6) ^ bit(j, 0)) << 2 | bit(j, 1) << 3 | bit(j, 2) << 4 |
           bit(j, 3) << 5 | bit(j, 6) << 6 | bit(j, 7) << 7;
  } else {
    return j;
  }
}
template <int P>
__device__ __forceinline__ int butterfly_of(int r) {
  if constexpr (P == 0) {
    return bit(r, 0) | bit(r, 1) << 1 | bit(r, 2) << 2 | bit(r, 5) << 3 | bit(r, 3) << 4 | bit(r, 4) << 5 |
           bit(r, 6) << 6 | bit(r, 7) << 7;
  } else if constexpr (P == 1) {
    return (bit(r, 2) ^ bit(r, 6)) | bit(r, 3) << 1 | bit(r, 4) << 2 | bit(r, 5) << 3 | bit(r, 0) << 4 |
           bit(r, 1) << 5 | bit(r, 6) << 6 | bit(r, 7) << 7;
  } else {
    return r;
  }
}

// A line's input read once: no L1 allocation (volatile keeps it ordered with
// the in-place stores).
__device__ __forceinline__ uint32_t ld_once_b32(const void* p) {
  uint32_t r;
  asm volatile("ld.global.L1::no_allocate.b32 %0, [%1];" : "=r"(r) : "l"(p));
  return r;
}
__device__ __forceinline__ uint16_t ld_once_b16(const void* p) {
  uint16_t r;
  asm volatile("ld.global.L1::no_allocate.b16 %0, [%1];" : "=h"(r) : "l"(p));
  return r;
}
__device__ __forceinline__ float2 ld_once_f2(const void* p) {
  float2 r;
  asm volatile("ld.global.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "l"(p));
  return r;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = uint64_t((addr >> 4) & 0x3FFF);
  d |= uint64_t((kLbo >> 4) & 0x3FFF) << 16;
  d |= uint64_t((kSbo >> 4) & 0x3FFF) << 32;
  d |= uint64_t(1) << 46;            // tcgen05 descriptor version
  return d;                          // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: FP32 accumulate, FP16 A and B, both
// K-major, N = 32, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t da, uint64_t db, bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(da), "l"(db), "r"(kIdesc), "r"(accumulate ? 1u : 0u)
      : "memory");
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

}  // namespace tc

// One radix-16 pass: MMA on the current A tile, then the D rows go either
// (P < 2) twiddled into the next A tile or (P == 2) to HBM.  Each thread owns
// TMEM lane tid of both M tiles (A/D rows tid and 128 + tid).  Returns false
// when the completion wait expired (all threads agree).
//
// Store addresses are a per-thread base plus a compile-time offset per q
// (t = j mod 16, rn = j / 16 for butterfly j; the pass-1 row map splits into
// the thread's bits and q's bits except row bit 2 = t2 ^ q0, hence the two
// bases for even and odd q).
//
// FILTER (last pass of a compression line's forward transform): instead of
// going to HBM, output q of butterfly j -- spectrum bin k = j + 256 q -- is
// multiplied by the filter H[k] in FP32, conjugated and shifted by 1/N
// (Eq. 1), and written as the inverse transform's pass-0 input: butterfly j
// of the inverse takes bins j + 256 r, so the 16 results form row rho_0(j)
// of A, four 16-byte stores.
// The MMAs of one pass on the A tile as the CTA's threads left it: barrier,
// four tcgen05.mma from one thread, commit, bounded wait.  Returns false
// when the wait expired (all threads agree); after true the accumulators
// may be read.
__device__ __forceinline__ bool tc_issue_wait(int* status, uint64_t* bar, uint32_t tmem, uint32_t a_base,
                                              uint32_t b_base, uint32_t& phase) {
  using namespace tc;
  fence_proxy_async_shared();
  fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    fence_after();
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int s = 0; s < 2; ++s)
        tc::mma(tmem + uint32_t(32 * t), tc::smem_desc(a_base + 8192 * t + 2 * kLbo * s),
                tc::smem_desc(b_base + 2 * kLbo * s), s > 0);
    tc::commit(bar);
  }
  const bool arrived = mbar_wait_bounded(bar, phase, status);
  if (__syncthreads_or(!arrived)) return false;
  phase ^= 1;
  fence_after();
  return true;
}

// Sixteen FP16 pairs x[r] as the pass-0 input of butterfly j (row rho_0(j),
// k-pairs r = 0..15): four 16-byte stores, conflict-free across a
// quarter-warp of consecutive j.
__device__ __forceinline__ void tc_store_row0(unsigned char* sA, int j, const uint32_t (&x)[16]) {
  using namespace tc;
  const int row = row_of<0>(j);
  unsigned char* dst = sA + (row >> 3) * kSbo + (row & 7) * 16;
#pragma unroll
  for (int c = 0; c < 4; ++c)
    *reinterpret_cast<uint4*>(dst + c * kLbo) = make_uint4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
}

// The last pass of a forward transform whose spectrum is filtered: output q
// of butterfly rho is bin k = rho + 256 q; conj(X[k] H[k]) / N (H conjugated
// first when CONJ_H) rounded to FP16 is the inverse's pass-0 input.
template <bool CONJ_H>
__device__ __forceinline__ void tc_filter_to_a(unsigned char* sA, int rho, const uint32_t (&d)[32],
                                               const float2* __restrict__ hk) {
  const float inv_n = 1.0f / float(tc::kN);
  uint32_t x[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    float2 h = __ldg(hk + 256 * q);
    if (CONJ_H) h.y = -h.y;
    const float2 y = cmul(make_float2(__uint_as_float(d[2 * q]), __uint_as_float(d[2 * q + 1])), h);
    const __half2 v = __floats2half2_rn(y.x * inv_n, -y.y * inv_n);
    x[q] = *reinterpret_cast<const uint32_t*>(&v);
  }
  tc_store_row0(sA, rho, x);
}

// FP8 storage (TOut an FP8 pair): the line's static block exponent,
// in_scale * out_scale (one of them is 1), scales the first pass's results in
// FP32 -- an exact power of two -- so the FP16 operands of the later passes
// stay in range and the last pass writes the stored scale directly.
template <int P, int MODE, bool FILTER = false, class TOut = __half2>
__device__ __forceinline__ bool tc_pass(const RowArgs& a, long long line, unsigned char* sA, uint64_t* bar,
                                        uint32_t tmem, uint32_t lane_tmem, uint32_t a_base, uint32_t b_base,
                                        uint32_t& phase, const float2* s_tw) {
  using namespace tc;
  constexpr bool kFp8 = !std::is_same<TOut, __half2>::value;
  const int tid = threadIdx.x;
  const float sc = kFp8 && P == 0 ? a.in_scale * a.out_scale : 1.0f;
  if (!tc_issue_wait(a.status, bar, tmem, a_base, b_base, phase)) return false;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t d[32];
    tc::ld32(lane_tmem + uint32_t(32 * h), d);
    const int rho = tid + 128 * h;
    const int j = tc::butterfly_of<P>(rho);
    if constexpr (P < 2) {
      const int t = j & 15, rn = j >> 4;
      const int rn_off = (rn >> 2) * kLbo + (rn & 3) * 4;
      int base_even, base_odd;
      const float2* tw_row = s_tw + rn * kTwPitch;       // W_256^{rn q}, q < 16 (rn = 0: ones)
      if constexpr (P == 0) {
        // Twiddles W_256^{rn q} from the shared-memory table: rows 144 B
        // apart put the four rn of a warp in four different 16-byte bank
        // groups; one 16-byte load fetches q and q + 1.
        const int t2 = (t >> 2) & 1;
        base_even = 16 * (t & 3) + 4160 * t2 + 8192 * (t >> 3) + rn_off;
        base_odd = base_even + 64 - 128 * t2;
        const float4* tw2 = reinterpret_cast<const float4*>(tw_row);
#pragma unroll
        for (int q2 = 0; q2 < 8; ++q2) {
          const float4 wp = tw2[q2];
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int q = 2 * q2 + e;
            const float2 w = e ? make_float2(wp.z, wp.w) : make_float2(wp.x, wp.y);
            float2 y = cmul(make_float2(__uint_as_float(d[2 * q]), __uint_as_float(d[2 * q + 1])), w);
            if constexpr (kFp8) y = cscale(y, sc);
            *reinterpret_cast<__half2*>(sA + (q & 1 ? base_odd : base_even) + 512 * (q >> 1)) =
                __float22half2_rn(y);
          }
        }
      } else {
        // Twiddles W_4096^{rn (t + 16 q)}: the geometric sequence from
        // W_4096^{rn t} with ratio W_256^{rn}, both read once (the sequence's
        // FP32 rounding, about 1e-6 after 15 steps, is far below the FP16
        // rounding of the operands it scales).
        base_even = 512 * (t >> 3) + 16 * (t & 7) + rn_off;
        float2 w = s_tw[(16 + rn) * kTwPitch + t];
        const float2 ratio = tw_row[1];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const float2 y = cmul(make_float2(__uint_as_float(d[2 * q]), __uint_as_float(d[2 * q + 1])), w);
          *reinterpret_cast<__half2*>(sA + base_even + 1024 * q) = __float22half2_rn(y);
          if (q < 15) w = cmul(w, ratio);
        }
      }
    } else if constexpr (FILTER) {
      tc_filter_to_a<false>(sA, rho, d, a.h + line * a.h_stride + rho);
    } else {
      // The inverse's final conjugation is folded into the last pass's matrix.
      TOut* out = static_cast<TOut*>(a.out) + line * a.out_stride + rho;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float2 y = make_float2(__uint_as_float(d[2 * q]), __uint_as_float(d[2 * q + 1]));
        if constexpr (kFp8) {
          Storage<TOut>::store(out + 256 * q, y);
        } else {
          out[256 * q] = __float22half2_rn(y);
        }
      }
      check_finite<Storage<TOut>, 16>(a.finite_flag, [&](int m) {
        return make_float2(__uint_as_float(d[2 * m]), __uint_as_float(d[2 * m + 1]));
      });
    }
  }
  fence_before();
  return true;
}

// CTA set-up shared by the tensor-core kernels: the three B matrices, the
// twiddle rows, the TMEM allocation (kTmemCols columns) and the mbarrier;
// returns the TMEM base address.
//   DFT-16 matrix in real form (prepared on the host in FP16, [n][k]) and two
//   derived copies for the inverse (Eq. 1 as conj(DFT(conj(x) / N))):
//     B_last  = B with the imaginary output rows n = 2 q + 1 negated (the
//               final conjugation);
//     B_first = B / N with the imaginary input columns k = 2 r + 1 negated
//               (the conjugated, 1/N-shifted input; N = 2^12 keeps every
//               coefficient normal in FP16, so the scaling is exact).
//   Twiddle rows from the pass-major table: [rn][q] = W_256^{rn q} (entry
//   16 (rn - 1) + q) and [16 + rn][t] = W_4096^{rn t} (entry
//   240 + 256 (rn - 1) + t), rn = 1..15, q, t < 16; the rows rn = 0 are ones.
__device__ __forceinline__ uint32_t tc_cta_setup(const void* tc_b, const float2* tw, unsigned char* smem) {
  using namespace tc;
  unsigned char* sB = smem + kBOff;
  float2* s_tw = reinterpret_cast<float2*>(smem + kTwOff);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kBarOff);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kBarOff + 8);
  const int tid = threadIdx.x, warp = tid >> 5;
  const __half* b_src = static_cast<const __half*>(tc_b);
  for (int i = tid; i < 32 * 32; i += kThreads) {
    const int n = i / 32, k = i % 32;
    const __half v = b_src[i];
    *reinterpret_cast<__half*>(sB + kmaj(n, k)) = v;
    *reinterpret_cast<__half*>(sB + kBBytes + kmaj(n, k)) = (n & 1) ? __hneg(v) : v;
    const __half vs = __float2half_rn(__half2float(v) * (1.0f / float(kN)));
    *reinterpret_cast<__half*>(sB + 2 * kBBytes + kmaj(n, k)) = (k & 1) ? __hneg(vs) : vs;
  }
  for (int i = tid; i < 2 * 256; i += kThreads) {
    const int tab = i / 256, rn = (i % 256) / 16, c = i % 16;
    s_tw[(16 * tab + rn) * kTwPitch + c] =
        rn == 0 ? make_float2(1.0f, 0.0f) : tw[tab == 0 ? 16 * (rn - 1) + c : 240 + 256 * (rn - 1) + c];
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) mbar_init(bar, 1);
  fence_proxy_async_shared();
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  fence_before();
  __syncthreads();
  fence_after();
  return *tslot;
}

// CTA teardown: a wait that expired leaves `phase` at the commit it was
// waiting for; that commit gets one more bounded wait before the tensor
// memory is freed.
__device__ __forceinline__ void tc_cta_teardown(bool ok, unsigned char* smem, uint32_t tmem, uint32_t phase) {
  using namespace tc;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kBarOff);
  if (!ok && threadIdx.x == 0) mbar_wait_bounded(bar, phase, nullptr);
  fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

// 128 threads per CTA, eight CTAs per SM: eight lines in flight per SM (the
// TMEM limit at 64 columns a line) while each CTA's passes run one after
// another.  Persistent: CTA b takes lines b, b + grid, ...; thread 0 bulk-
// prefetches the CTA's next line into L2.
template <int MODE, class TIn, class TOut = __half2>
__global__ void __launch_bounds__(tc::kThreads, tc::kCtasPerSm) fft_tc_kernel(const RowArgs a) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  unsigned char* sA = smem_tc;
  unsigned char* sB = smem_tc + kBOff;
  float2* s_tw = reinterpret_cast<float2*>(smem_tc + kTwOff);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_tc + kBarOff);
  const int tid = threadIdx.x, warp = tid >> 5;
  const TIn* in_lines = static_cast<const TIn*>(a.in);

  const uint32_t tmem = tc_cta_setup(a.tc_b, a.tw, smem_tc);
  const uint32_t lane_tmem = tmem + (uint32_t(32 * warp) << 16);
  const uint32_t a_base = smem_addr(sA), b_base = smem_addr(sB);
  const uint32_t b_first = MODE == kInverse ? b_base + 2 * kBBytes : b_base;
  const uint32_t b_last = MODE != kForward ? b_base + kBBytes : b_base;
  uint32_t phase = 0;
  bool ok = true;

  for (long long line = blockIdx.x; ok && line < a.lines; line += gridDim.x) {
    const long long next = line + gridDim.x;
    if (a.pf_ahead > 0 && tid == 0 && next < a.lines)   // next iteration's line, into L2
      prefetch_l2_bulk(in_lines + next * a.in_stride, uint32_t(kN * sizeof(TIn)));
    // Pass-0 inputs: butterfly j takes x[j + 256 r]; its row of A is four
    // 16-byte core-matrix rows, one st.shared.v4 per four points (the eight
    // lanes of a quarter-warp have distinct row % 8).  Complex64 inputs are
    // rounded to FP16 operands here; FP8 pairs convert exactly.
    const TIn* in = in_lines + line * a.in_stride + tid;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = tid + 128 * h;
      uint32_t x[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        if constexpr (sizeof(TIn) == 4) {
          x[r] = ld_once_b32(in + 128 * h + 256 * r);
        } else if constexpr (sizeof(TIn) == 2) {
          const __half2_raw v = __nv_cvt_fp8x2_to_halfraw2(
              __nv_fp8x2_storage_t(ld_once_b16(in + 128 * h + 256 * r)), Fp8Format<TIn>::kInterp);
          x[r] = uint32_t(v.x) | (uint32_t(v.y) << 16);
        } else {
          const __half2 v = __float22half2_rn(ld_once_f2(in + 128 * h + 256 * r));
          x[r] = *reinterpret_cast<const uint32_t*>(&v);
        }
      }
      tc_store_row0(sA, j, x);
    }
    if constexpr (MODE == kCompress) {
      // Forward, filter (into A, conjugated and shifted), inverse: the inverse's
      // input is already conj(Y) / N, so its first pass takes plain B.
      ok = tc_pass<0, MODE>(a, line, sA, bar, tmem, lane_tmem, a_base, b_base, phase, s_tw) &&
           tc_pass<1, MODE>(a, line, sA, bar, tmem, lane_tmem, a_base, b_base, phase, s_tw) &&
           tc_pass<2, MODE, true>(a, line, sA, bar, tmem, lane_tmem, a_base, b_base, phase, s_tw) &&
           tc_pass<0, MODE>(a, line, sA, bar, tmem, lane_tmem, a_base, b_base, phase, s_tw) &&
           tc_pass<1, MODE>(a, line, sA, bar, tmem, lane_tmem, a_base, b_base, phase, s_tw) &&
           tc_pass<2, MODE>(a, line, sA, bar, tmem, lane_tmem, a_base, b_last, phase, s_tw);
    } else {
      ok = tc_pass<0, MODE, false, TOut>(a, line, sA, bar, tmem, lane_tmem, a_base, b_first, phase, s_tw) &&
           tc_pass<1, MODE, false, TOut>(a, line, sA, bar, tmem, lane_tmem, a_base, b_base, phase, s_tw) &&
           tc_pass<2, MODE, false, TOut>(a, line, sA, bar, tmem, lane_tmem, a_base, b_last, phase, s_tw);
    }
  }
  tc_cta_teardown(ok, smem_tc, tmem, phase);
}

template <int MODE, class TIn, class TOut = __half2>
cudaError_t launch_tc_kernel(const RowArgs& a, cudaStream_t stream) {
  auto kern = fft_tc_kernel<MODE, TIn, TOut>;
  // kCtasPerSm CTAs per SM: the register limit of __launch_bounds__; tensor
  // memory holds exactly that many 64-column allocations, so the persistent
  // CTAs never wait on each other's allocation.  Computed once,
  // thread-safely (function-local static).
  static const LaunchSetup setup = []() -> LaunchSetup {
    LaunchSetup r{cudaSuccess, 0};
    int dev = 0, sms = 0;
    if ((r.err = cudaGetDevice(&dev)) != cudaSuccess) return r;
    if ((r.err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return r;
    r.resident = tc::kCtasPerSm * sms;
    return r;
  }();
  if (setup.err != cudaSuccess) return setup.err;
  (void)kern;
  if (a.lines <= 0) return cudaSuccess;
  const int grid = int(a.lines < setup.resident ? a.lines : setup.resident);
  RowArgs b = a;
  b.pf_ahead = a.no_prefetch ? 0 : 1;       // dense rows in device memory: prefetch the next line
  kern<<<grid, tc::kThreads, tc::kSmemBytes, stream>>>(b);
  return cudaGetLastError();
}

template <class TS, int MODE>
cudaError_t launch_tc_n(const RowArgs& a, cudaStream_t stream) {
  static_assert(sizeof(TS) == sizeof(__half2), "the tensor-core rows take FP16 storage");
  return launch_tc_kernel<MODE, __half2>(a, stream);
}

}  // namespace bfp
