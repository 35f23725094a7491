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
// Rows: butterfly j of pass p sits in A/D row rho_p(j); thread tau (TMEM lane
// tau % 128 of tile tau / 128) handles the butterfly in row tau.  rho_p keep
// every shared-memory store of the producer free of bank conflicts (below).
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
constexpr int kLbo = 128;            // bytes between K-adjacent core matrices
constexpr int kSbo = 512;            // bytes between 8-row groups (4 core matrices of K = 32)
constexpr int kABytes = kB * 64;     // 256 rows x 32 FP16
constexpr int kBBytes = 32 * 64;     // 32 rows x 32 FP16
constexpr int kSmemBytes = kABytes + kBBytes + 16;
constexpr uint32_t kTmemCols = 64;   // two 128 x 32 FP32 accumulators

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
// and the pass-0 loads visit the k-pairs in a lane-rotated order.
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

__device__ __forceinline__ void store_pair(unsigned char* sA, int row, int r, float2 v) {
  *reinterpret_cast<__half2*>(sA + kmaj(row, 2 * r)) = __float22half2_rn(v);
}

}  // namespace tc

// One radix-16 pass: MMA on the current A tile, then the D rows go either
// (P < 2) twiddled into the next A tile or (P == 2) to HBM.  Returns false
// when the completion wait expired (all threads agree).
template <int P, class TS, int MODE>
__device__ __forceinline__ bool tc_pass(const RowArgs& a, long long line, unsigned char* sA, uint64_t* bar,
                                        uint32_t tmem, uint32_t my_tmem, uint32_t a_base, uint32_t b_base,
                                        uint32_t& phase) {
  using namespace tc;
  const int tid = threadIdx.x;
  fence_proxy_async_shared();
  fence_before();
  __syncthreads();
  if (tid == 0) {
    fence_after();
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int s = 0; s < 2; ++s)
        tc::mma(tmem + uint32_t(32 * t), tc::smem_desc(a_base + 8192 * t + 2 * kLbo * s),
                tc::smem_desc(b_base + 2 * kLbo * s), s > 0);
    tc::commit(bar);
  }
  const bool arrived = mbar_wait_bounded(bar, phase, a.status);
  if (__syncthreads_or(!arrived)) return false;
  phase ^= 1;
  fence_after();
  uint32_t d[32];
  tc::ld32(my_tmem, d);
  const int j = tc::butterfly_of<P>(tid);
  if constexpr (P < 2) {
    constexpr int kLogNs = 4 * P;                      // sub-length 16^P of this pass
    constexpr int kNs2 = 16 << kLogNs;                 // sub-length of the next pass
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int i = ((j >> kLogNs) << (kLogNs + 4)) + (j & ((1 << kLogNs) - 1)) + (q << kLogNs);
      const int jn = i & 255, rn = i >> 8;
      float2 y = make_float2(__uint_as_float(d[2 * q]), __uint_as_float(d[2 * q + 1]));
      if (rn > 0) y = cmul(y, __ldg(a.tw + (kNs2 - 16) + (rn - 1) * kNs2 + (jn & (kNs2 - 1))));
      tc::store_pair(sA, tc::row_of<P + 1>(jn), rn, y);
    }
  } else {
    TS* out = static_cast<TS*>(a.out) + line * a.out_stride + j;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      float2 y = make_float2(__uint_as_float(d[2 * q]), __uint_as_float(d[2 * q + 1]));
      if (MODE == kInverse) y = cconj(y);
      Storage<TS>::store(out + 256 * q, y);
    }
    check_finite<Storage<TS>, 16>(a.finite_flag, [&](int m) {
      return make_float2(__uint_as_float(d[2 * m]), __uint_as_float(d[2 * m + 1]));
    });
  }
  fence_before();
  return true;
}

template <class TS, int MODE>
__global__ void __launch_bounds__(256, 3) fft_tc_kernel(const RowArgs a) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  unsigned char* sA = smem_tc;
  unsigned char* sB = smem_tc + kABytes;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_tc + kABytes + kBBytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem_tc + kABytes + kBBytes + 8);
  const int tid = threadIdx.x, warp = tid >> 5;
  const float inv_n = 1.0f / float(kN);

  // DFT-16 matrix in real form (prepared on the host in FP16, [n][k]).
  const __half* b_src = static_cast<const __half*>(a.tc_b);
  for (int i = tid; i < 32 * 32; i += 256) *reinterpret_cast<__half*>(sB + kmaj(i / 32, i % 32)) = b_src[i];
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
  const uint32_t tmem = *tslot;
  const uint32_t my_tmem = tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(32 * (warp >> 2));
  const uint32_t a_base = smem_addr(sA), b_base = smem_addr(sB);
  uint32_t phase = 0;
  bool ok = true;

  for (long long line = blockIdx.x; ok && line < a.lines; line += gridDim.x) {
    if (a.pf_ahead > 0 && tid == 0 && line + gridDim.x < a.lines)   // next iteration's line, into L2
      prefetch_l2_bulk(static_cast<const TS*>(a.in) + (line + gridDim.x) * a.in_stride, uint32_t(kN * sizeof(TS)));
    // Pass-0 inputs: butterfly j = tid takes x[j + 256 r]; coalesced loads.
    const TS* in = static_cast<const TS*>(a.in) + line * a.in_stride + tid;
    const int row = tc::row_of<0>(tid);
    const int rot = (tid >> 3) & 3;                     // lane-rotated k-pair order
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int r = (m + rot) & 15;
      float2 x = Storage<TS>::load(in + 256 * r);
      if (MODE == kInverse) x = cscale(cconj(x), inv_n);
      tc::store_pair(sA, row, r, x);
    }
    ok = tc_pass<0, TS, MODE>(a, line, sA, bar, tmem, my_tmem, a_base, b_base, phase) &&
         tc_pass<1, TS, MODE>(a, line, sA, bar, tmem, my_tmem, a_base, b_base, phase) &&
         tc_pass<2, TS, MODE>(a, line, sA, bar, tmem, my_tmem, a_base, b_base, phase);
  }
  // A wait that expired leaves `phase` at the commit it was waiting for:
  // give that commit one more bounded wait before the tensor memory goes.
  if (!ok && tid == 0) mbar_wait_bounded(bar, phase, nullptr);
  fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

template <class TS, int MODE>
cudaError_t launch_tc_n(const RowArgs& a, cudaStream_t stream) {
  auto kern = fft_tc_kernel<TS, MODE>;
  // Three CTAs per SM: the register limit of __launch_bounds__(256, 3);
  // tensor memory would allow eight (64 of 512 columns each), so the
  // persistent CTAs never wait on each other's allocation.  Computed once,
  // thread-safely (function-local static).
  static const LaunchSetup setup = []() -> LaunchSetup {
    LaunchSetup r{cudaSuccess, 0};
    int dev = 0, sms = 0;
    if ((r.err = cudaGetDevice(&dev)) != cudaSuccess) return r;
    if ((r.err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return r;
    r.resident = 3 * sms;
    return r;
  }();
  if (setup.err != cudaSuccess) return setup.err;
  const int grid_cap = setup.resident;
  (void)kern;
  if (a.lines <= 0) return cudaSuccess;
  const int grid = int(a.lines < grid_cap ? a.lines : grid_cap);
  RowArgs b = a;
  b.pf_ahead = a.no_prefetch ? 0 : 1;       // dense rows in device memory: prefetch the next line
  kern<<<grid, 256, tc::kSmemBytes, stream>>>(b);
  return cudaGetLastError();
}

}  // namespace bfp
