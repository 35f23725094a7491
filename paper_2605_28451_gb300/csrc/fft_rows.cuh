// Batched row transforms: one length-N line per thread group, all passes on chip.
//
// Method (Sections III-B, IV and V of the paper, re-designed for sm_103a):
//
//   forward   X = DFT(x)                                   (unnormalised)
//   inverse   y = conj(DFT(conj(z) * 1/N))                 (Eq. 1: the 1/N block
//                                                           shift folded into the
//                                                           pre-inverse conjugate)
//   compress  y = conj(DFT(conj(DFT(x) . H) * 1/N))        (matched filter,
//                                                           Section III-B, Fig. 1)
//
// and the naive schedule of Section III-B, which drops the shift, stores the
// unnormalised inverse to FP16 and only then scales by 1/N.
//
// Layout.  Lines are rows of N interleaved complex points, consecutive lines
// `stride` points apart.  A group of T = N/16 threads owns one line; thread t
// holds the 16 points x[t + T m], m = 0..15, in FP32 registers.  Loads and
// stores of one warp touch consecutive points (coalesced), so every line is
// read from HBM once and written once.
//
// Passes.  Stockham autosort, radix 16 for every pass but possibly the last
// (radix 2, 4 or 8 when log2 N is not a multiple of 4).  A pass with radix R
// and current sub-length Ns takes butterfly j = t + T b (b < 16/R) over the
// points x[j + r N/R], multiplies point r by W_{Ns R}^{(j mod Ns) r}, runs the
// R-point DFT in registers and writes point r to y[(j / Ns) Ns R + j mod Ns +
// r Ns].  Between passes the line goes through shared memory in FP32 (one slot
// of padding every 16 points keeps the stride-16 writes of the first pass free
// of bank conflicts); after the last pass thread t holds X[t + T m] again, so
// the forward result of a compress feeds the inverse without an exchange.
//
// Corner turns.  With TLOAD / TSTORE a line is a column of a row-major matrix
// (point k of line l at k * stride + l).  The CTAs of a thread-block cluster
// then move 8 lines at a time: each CTA reads (or writes) a slab of k for all
// 8 lines as 32-byte segments and exchanges the points with the owning CTA
// through distributed shared memory, so a transpose costs no extra HBM pass.
//
// Twiddles come from a per-length FP32 table generated on the GPU in FP64
// (sincospi) and rounded once -- never by recurrence, which the paper
// identifies as the source of the ~42 dB "pure FP16" figure (Section III-A).
// The table is pass-major: for every pass after the first (sub-length Ns,
// radix R) it holds W_{Ns R}^{k r} at offset (Ns - 16) + (r - 1) Ns + k,
// r in [1, R), k in [0, Ns); N - 16 entries in all.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "async_copy.cuh"
#include "complex_ops.cuh"
#include "storage.cuh"

namespace bfp {

enum RowMode : int { kForward = 0, kInverse = 1, kCompress = 2 };

struct RowArgs {
  const void* in;
  void* out;
  const float2* tw;        // W_N^i for i in [0, N), FP32
  const float2* h;         // filter spectrum [N] (compress only)
  long long h_stride;      // compress: points between the filters of consecutive lines (0: one filter for all)
  long long lines;         // number of lines
  long long in_stride;     // points between consecutive input lines
  long long out_stride;    // points between consecutive output lines
  float in_scale;          // applied to loaded values (FP8 block exponent)
  float out_scale;         // applied before the final rounding (FP8 block exponent)
  int* status;             // device status word (bounded waits record timeouts here)
  int variant;             // RowVariant
  const float2* tw_line;   // N >= 8192: pass-major table of the 4096-point row transforms
  const float2* tw_4step;  // N >= 8192: four-step twiddles T[k1][n2] = W_N^{n2 k1}
  const void* tc_b;        // tensor-core variant: 16-point DFT matrix, real form, FP16 [32][32]
  int pf_ahead;            // > 0: each CTA prefetches into L2 the lines of the CTA pf_ahead blocks later
  int no_prefetch;         // nonzero: the input is not device memory; no bulk L2 prefetch of it
  int* finite_flag;        // non-null: dense-row stores record non-finite outputs here (BFPFFT_CHECK_FINITE)
  const void* tw16;        // 16-bit arithmetic rows: pass-major table of (w, -i conj w) 16-bit pairs
  int fs_h16;              // FP16 storage, lines of 8192 points or more by the four-step kernel: nonzero sends
                           // the row exchange between the column and row transforms as FP16 words
  const int* in_exp;       // adaptive exponents: per-line input exponents (value = stored * 2^e), or null
  int* out_exp;            // adaptive exponents: per-line output exponents written by the kernel
  const long long* line_off;   // non-null: line l starts at point line_off[l] of both in and out (the lines
                               // of one length in an uneven batch); dense rows of the plain and generic row
                               // kernels and of the four-step kernel only.  Offsets are multiples of 16 points.
};

// First point of a dense line: at line_off[line] when the lines are listed,
// else at line * stride.
__device__ __forceinline__ long long line_start(const RowArgs& a, long long line, long long stride) {
  return a.line_off != nullptr ? a.line_off[line] : line * stride;
}

// Row-kernel variants for dense rows of length <= 4096 (chosen by
// BFPFFT_ROWS or the tuner): bulk-copy pipelined persistent kernel or plain
// one-group-per-CTA kernel, with an FP32 or FP16 shared-memory exchange in
// one buffer or two (ping-pong), at 3 or 4 CTAs per SM, with or without a
// bulk L2 prefetch of the lines of the CTA one resident wave later (_l2).
// FP16 exchanges apply to FP16 storage only.  Shapes a variant does not
// cover run the pipelined kernel (TMA family) or the generic kernel (the
// rest; the _l2 prefetch applies there too when rows are dense).
enum RowVariant : int {
  kRowsTma = 0, kRowsPlain = 1, kRowsPlainPP = 2, kRowsPlainH = 3, kRowsPlainHPP = 4,
  kRowsTmaPP = 5, kRowsTmaH = 6, kRowsTmaHPP = 7, kRowsTc = 8, kRowsPlain4 = 9,
  kRowsPlainL2 = 10, kRowsPlain4L2 = 11, kRowsPlainHL2 = 12, kRowsPlainH4L2 = 13, kRowsPlainHS4L2 = 14,
  kRowsTwoPass = 15   // lines of 32768 and 65536 points: two streaming passes (twopass.cu) instead of four-step
};

constexpr int kPointsPerThread = 16;

#ifndef BFP_MIN_BLOCKS
#define BFP_MIN_BLOCKS 3
#endif

__host__ __device__ constexpr int pad16(int i) { return i + (i >> 4); }

template <int N, bool TURN = false>
struct RowShape {
  static constexpr int P = kPointsPerThread;
  static constexpr int T = N / P;                        // threads per line
  static constexpr int kThreads = N <= 4096 ? 256 : T;   // threads per CTA
  static constexpr int G = kThreads / T;                 // lines per CTA
  // Corner-turn kernels stage whole lines in shared memory even for N = 16.
  static constexpr int kSmemPerLine = (N > 16 || TURN) ? pad16(N) : 0;   // float2 slots
  static constexpr size_t kSmemBytes = size_t(G) * kSmemPerLine * sizeof(float2);
  // Cluster size of a corner-turn kernel: enough CTAs for 8 lines.
  static constexpr int C = TURN ? (G >= 8 ? 1 : 8 / G) : 1;
  static constexpr int kLinesPerCluster = C * G;
  // Resident CTAs per SM requested from the register allocator.
  static constexpr int kMinBlocks = kThreads >= 1024 ? 1 : (kThreads >= 512 ? 1 : BFP_MIN_BLOCKS);
  // Dense-row (no corner turn) kernels: 64 registers, so 4 CTAs per SM of 256
  // threads (faster than 3 at 80 in every mode; spills stay within 16 bytes)
  // and 2 of 512 (N = 8192).
  static constexpr int kMinBlocksDense = TURN ? kMinBlocks : (kThreads >= 1024 ? 1 : (kThreads >= 512 ? 2 : 4));
};

// Where a line lives between passes.  Every policy offers load / store of
// point i for exchange number Q (Q = 0 after the first pass, 1 after the
// second, ...), a barrier after the stores (sync) and a barrier before the
// next stores may overwrite what was just loaded (sync_war).
//
//   LocalXch          this CTA's shared memory, FP32, one buffer
//   LocalXchPP        FP32, two buffers used alternately: the next pass writes
//                     the other buffer, so no barrier is needed before it
//   LocalXchH         FP16 (half2) in shared memory: the paper's own layout
//                     (Section V: half2 threadgroup memory); every exchange is
//                     an FP16 storage point, so the inverse relies on the 1/N
//                     shift (Eq. 1) to keep intermediates in range
//   LocalXchHPP       FP16, two buffers
//   ClusterXch<SLAB>  a line spread over the CTAs of a thread-block cluster,
//                     SLAB points per CTA, through distributed shared memory
struct LocalXch {
  float2* sm;
  template <int Q> __device__ __forceinline__ float2 load(int i) const { return sm[pad16(i)]; }
  template <int Q> __device__ __forceinline__ void store(int i, float2 v) const { sm[pad16(i)] = v; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ void sync_war() const { __syncthreads(); }
};

template <int LINE>   // padded slots of one buffer
struct LocalXchPP {
  float2* sm;
  template <int Q> __device__ __forceinline__ float2 load(int i) const { return sm[(Q & 1) * LINE + pad16(i)]; }
  template <int Q> __device__ __forceinline__ void store(int i, float2 v) const { sm[(Q & 1) * LINE + pad16(i)] = v; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ void sync_war() const {}
};

struct LocalXchH {
  __half2* sm;
  template <int Q> __device__ __forceinline__ float2 load(int i) const { return __half22float2(sm[pad16(i)]); }
  template <int Q> __device__ __forceinline__ void store(int i, float2 v) const { sm[pad16(i)] = __float22half2_rn(v); }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ void sync_war() const { __syncthreads(); }
};

// FP16 exchange without padding: the slot of point i is i XOR h(i >> 5) on
// its low five bits, h(q) = (q & 15) | (bit 3 of q) << 4, which makes the
// stride-16 stores of the first pass, the 256-apart half-warps of the second
// and the consecutive loads free of bank conflicts for every length from 256
// (with 4-byte slots, where one padding slot per 16 leaves a two-way conflict
// on every consecutive load).
__host__ __device__ constexpr int swz32(int i) { return i ^ (((i >> 5) & 15) | ((((i >> 5) >> 3) & 1) << 4)); }

struct LocalXchHS {
  __half2* sm;
  template <int Q> __device__ __forceinline__ float2 load(int i) const { return __half22float2(sm[swz32(i)]); }
  template <int Q> __device__ __forceinline__ void store(int i, float2 v) const { sm[swz32(i)] = __float22half2_rn(v); }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ void sync_war() const { __syncthreads(); }
};

template <int LINE>
struct LocalXchHPP {
  __half2* sm;
  template <int Q> __device__ __forceinline__ float2 load(int i) const {
    return __half22float2(sm[(Q & 1) * LINE + pad16(i)]);
  }
  template <int Q> __device__ __forceinline__ void store(int i, float2 v) const {
    sm[(Q & 1) * LINE + pad16(i)] = __float22half2_rn(v);
  }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ void sync_war() const {}
};

template <int SLAB>
struct ClusterXch {
  float2* base;   // this CTA's slab (same offset in every CTA of the cluster)
  __device__ __forceinline__ float2* at(int i) const {
    return cooperative_groups::this_cluster().map_shared_rank(base + pad16(i % SLAB), i / SLAB);
  }
  template <int Q> __device__ __forceinline__ float2 load(int i) const { return *at(i); }
  template <int Q> __device__ __forceinline__ void store(int i, float2 v) const { *at(i) = v; }
  __device__ __forceinline__ void sync() const { cooperative_groups::this_cluster().sync(); }
  __device__ __forceinline__ void sync_war() const { cooperative_groups::this_cluster().sync(); }
};

__host__ __device__ constexpr int ilog16(int ns) { return ns <= 1 ? 0 : 1 + ilog16(ns / 16); }

// Exchange variants of the single-CTA row kernels.
enum XchVariant : int { kXchF32 = 0, kXchF32PP = 1, kXchF16 = 2, kXchF16PP = 3, kXchF16S = 4 };

template <int N, int XV> struct XchSel;
template <int N> struct XchSel<N, kXchF32> {
  static constexpr size_t kLineBytes = size_t(N > 16 ? pad16(N) : 0) * sizeof(float2);
  __device__ __forceinline__ static LocalXch make(unsigned char* p) { return LocalXch{reinterpret_cast<float2*>(p)}; }
};
template <int N> struct XchSel<N, kXchF32PP> {
  static constexpr size_t kLineBytes = 2 * size_t(pad16(N)) * sizeof(float2);
  __device__ __forceinline__ static LocalXchPP<pad16(N)> make(unsigned char* p) {
    return LocalXchPP<pad16(N)>{reinterpret_cast<float2*>(p)};
  }
};
template <int N> struct XchSel<N, kXchF16> {
  static constexpr size_t kLineBytes = size_t(pad16(N)) * sizeof(__half2);
  __device__ __forceinline__ static LocalXchH make(unsigned char* p) { return LocalXchH{reinterpret_cast<__half2*>(p)}; }
};
template <int N> struct XchSel<N, kXchF16S> {
  static constexpr size_t kLineBytes = size_t(N) * sizeof(__half2);
  __device__ __forceinline__ static LocalXchHS make(unsigned char* p) { return LocalXchHS{reinterpret_cast<__half2*>(p)}; }
};
template <int N> struct XchSel<N, kXchF16PP> {
  static constexpr size_t kLineBytes = 2 * size_t(pad16(N)) * sizeof(__half2);
  __device__ __forceinline__ static LocalXchHPP<pad16(N)> make(unsigned char* p) {
    return LocalXchHPP<pad16(N)>{reinterpret_cast<__half2*>(p)};
  }
};

template <int N, int Ns>
struct StockhamPass {
  static constexpr int P = kPointsPerThread;
  static constexpr int T = N / P;
  static constexpr int R = (N / Ns) >= 16 ? 16 : N / Ns;
  static constexpr int B = P / R;
  static constexpr bool kLast = (Ns * R == N);
  static constexpr int kQ = ilog16(Ns);   // exchange number written by this pass

  template <class X>
  __device__ __forceinline__ static void run(float2 (&v)[P], const float2* __restrict__ tw, const X& x, int t) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = t + T * b;
      const int k = j & (Ns - 1);
      float2 u[R];
#pragma unroll
      for (int r = 0; r < R; ++r) u[r] = v[b + B * r];
      if (Ns > 1) {
        // Pass-major table: W_{Ns R}^{k r} at (Ns - 16) + (r - 1) Ns + k, so the
        // lanes of a warp (consecutive k) read consecutive twiddles.
        const float2* twp = tw + (Ns - 16) + k;
#pragma unroll
        for (int r = 1; r < R; ++r) u[r] = cmul(u[r], __ldg(twp + (r - 1) * Ns));
      }
      Dft<R>::run(u);
      if (kLast) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[b + B * r] = u[r];
      } else {
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) x.template store<kQ>(base + r * Ns, u[r]);
      }
    }
    if constexpr (!kLast) {
      x.sync();
#pragma unroll
      for (int m = 0; m < P; ++m) v[m] = x.template load<kQ>(t + T * m);
      x.sync_war();
      StockhamPass<N, Ns * R>::run(v, tw, x, t);
    }
  }
};

// Full forward DFT of the line held in v (v[m] = x[t + T m] -> X[t + T m]).
template <int N, class X>
__device__ __forceinline__ void line_dft(float2 (&v)[kPointsPerThread], const float2* __restrict__ tw,
                                         const X& x, int t) {
  StockhamPass<N, 1>::run(v, tw, x, t);
}

template <int N>
__device__ __forceinline__ void line_dft(float2 (&v)[kPointsPerThread], const float2* __restrict__ tw,
                                         float2* __restrict__ sm, int t) {
  StockhamPass<N, 1>::run(v, tw, LocalXch{sm}, t);
}

// The per-line chain between load and store: block exponents, the inverse's
// conj * 1/N (Eq. 1), the transform(s), the filter multiply of compress mode,
// the final conjugate, and the naive FP16 rounding of Section III-B.
template <int N, int MODE, bool NAIVE, bool SCALED, class X = LocalXch>
__device__ __forceinline__ void row_compute_x(float2 (&v)[kPointsPerThread], const RowArgs& a, const X& xch, int t,
                                              long long line = 0);

template <int N, int MODE, bool NAIVE, bool SCALED>
__device__ __forceinline__ void row_compute(float2 (&v)[kPointsPerThread], const RowArgs& a, float2* sm, int t,
                                            long long line = 0) {
  row_compute_x<N, MODE, NAIVE, SCALED>(v, a, LocalXch{sm}, t, line);
}

template <int N, int MODE, bool NAIVE, bool SCALED, class X>
__device__ __forceinline__ void row_compute_x(float2 (&v)[kPointsPerThread], const RowArgs& a, const X& xch, int t,
                                              long long line) {
  constexpr int P = kPointsPerThread, T = N / P;
  const float inv_n = 1.0f / float(N);
  if (SCALED) {
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = cscale(v[m], a.in_scale);
  }
  if (MODE == kInverse) {
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = NAIVE ? cconj(v[m]) : cscale(cconj(v[m]), inv_n);
  }

  line_dft<N>(v, a.tw, xch, t);

  if (MODE == kCompress) {
    // This line's filter (idle groups past the last line read line 0's).
    const float2* hl = a.h + (line < a.lines ? line : 0) * a.h_stride;
    // Filter loads in groups of four: keeps the compiler from hoisting all
    // sixteen next to the line (register pressure at 3 CTAs / SM).
#pragma unroll
    for (int m0 = 0; m0 < P; m0 += 4) {
      float2 h[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) h[i] = __ldg(hl + t + T * (m0 + i));
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 p = cmul(v[m0 + i], h[i]);
        v[m0 + i] = NAIVE ? cconj(p) : cscale(cconj(p), inv_n);
      }
      asm volatile("" ::: "memory");
    }
    // An opaque copy of t keeps the compiler from holding the first
    // transform's address arithmetic live for reuse in the second.
    int t2;
    asm volatile("mov.b32 %0, %1;" : "=r"(t2) : "r"(t));
    line_dft<N>(v, a.tw, xch, t2);
  }
  if (MODE == kInverse || MODE == kCompress) {
#pragma unroll
    for (int m = 0; m < P; ++m) {
      v[m] = cconj(v[m]);
      if (NAIVE) v[m] = naive_half_then_scale(v[m], inv_n);
    }
  }
  if (SCALED) {
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = cscale(v[m], a.out_scale);
  }
}

// Pointer to slot `idx` of line `l` of the cluster (l in [0, kLinesPerCluster)).
template <class S>
__device__ __forceinline__ float2* cluster_slot(float2* local_base, int l, int idx) {
  float2* p = local_base + (l % S::G) * S::kSmemPerLine + idx;
  if constexpr (S::C > 1) {
    return cooperative_groups::this_cluster().map_shared_rank(p, l / S::G);
  } else {
    return p;
  }
}

// Load of slot `idx` of line `l` of the cluster: ld.shared::cluster through
// mapa for a peer's row buffer, a plain shared load when C == 1.
template <class S>
__device__ __forceinline__ float2 cluster_load(float2* local_base, int l, int idx) {
  float2* p = local_base + (l % S::G) * S::kSmemPerLine + idx;
  if constexpr (S::C > 1) {
    const uint32_t addr = mapa(smem_addr(p), uint32_t(l / S::G));
    float2 r;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "r"(addr) : "memory");
    return r;
  } else {
    return *p;
  }
}

template <class S>
__device__ __forceinline__ void cluster_store(float2* local_base, int l, int idx, float2 v) {
  float2* p = local_base + (l % S::G) * S::kSmemPerLine + idx;
  if constexpr (S::C > 1) {
    const uint32_t addr = mapa(smem_addr(p), uint32_t(l / S::G));
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
  } else {
    *p = v;
  }
}

template <class S>
__device__ __forceinline__ void cluster_barrier() {
  if constexpr (S::C > 1) {
    cooperative_groups::this_cluster().sync();
  } else {
    __syncthreads();
  }
}

template <int N, class TIn, class TOut, int MODE, bool NAIVE, bool SCALED, bool TLOAD, bool TSTORE, int XV = kXchF32,
          int MINB = 0>
__global__ void __launch_bounds__(RowShape<N, TLOAD || TSTORE>::kThreads,
                                  MINB > 0 ? MINB : RowShape<N, TLOAD || TSTORE>::kMinBlocksDense)
fft_rows_kernel(const RowArgs a) {
  static_assert(XV == kXchF32 || (!TLOAD && !TSTORE), "corner turns stage lines in FP32");
  using S = RowShape<N, TLOAD || TSTORE>;
  constexpr int P = S::P, T = S::T;
  extern __shared__ float2 smem_rows[];
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const long long line = (long long)blockIdx.x * S::G + g;
  const bool active = line < a.lines;
  float2* sm = smem_rows + g * S::kSmemPerLine;
  // First line of this CTA's cluster (clusters are runs of C consecutive CTAs).
  const long long line0 = (long long)(blockIdx.x / S::C) * S::kLinesPerCluster;
  const int rank = int(blockIdx.x % S::C);
  constexpr int kSlab = N / S::C;                        // points per CTA in a corner turn

  float2 v[P];
  if constexpr (TLOAD) {
    // Gather: this CTA reads points [rank * kSlab, (rank + 1) * kSlab) of all
    // cluster lines and writes each line's values into the row buffer of the
    // CTA that transforms it.  With 8 lines per cluster a thread owns two
    // points and reads each point's 8 lines as one contiguous segment (32 B in
    // FP16), so a warp's remote stores go to one CTA, 32 consecutive points.
    static_assert(kSlab * S::kLinesPerCluster == P * S::kThreads, "one slot per thread and point");
    const TIn* in = static_cast<const TIn*>(a.in);
    if constexpr (S::kLinesPerCluster == 8 && std::is_same<TIn, __half2>::value) {
      // FP16 input moves as raw half2 words (exact): half the bytes.
      constexpr int Q = kSlab / S::kThreads;
      const bool seg = line0 + 8 <= a.lines && a.in_stride % 4 == 0;
      uint32_t x[Q][8];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int k = rank * kSlab + int(threadIdx.x) + S::kThreads * q;
        const __half2* src = in + (long long)k * a.in_stride + line0;
        if (seg) {
          seg8_load_raw(src, x[q]);
        } else {
#pragma unroll
          for (int l = 0; l < 8; ++l)
            x[q][l] = line0 + l < a.lines ? __ldcs(reinterpret_cast<const unsigned int*>(src + l)) : 0u;
        }
      }
      cluster_barrier<S>();
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int k = rank * kSlab + int(threadIdx.x) + S::kThreads * q;
#pragma unroll
        for (int l = 0; l < 8; ++l) {
          // Line l's row buffer, read as 32-bit words (the first half of it).
          uint32_t* slot = reinterpret_cast<uint32_t*>(smem_rows + (l % S::G) * S::kSmemPerLine) + pad16(k);
          if constexpr (S::C > 1) {
            st_cluster_b32(mapa(smem_addr(slot), uint32_t(l / S::G)), x[q][l]);
          } else {
            *slot = x[q][l];
          }
        }
      }
    } else if constexpr (S::kLinesPerCluster == 8) {
      constexpr int Q = kSlab / S::kThreads;   // points per thread (2)
      const bool seg = line0 + 8 <= a.lines && a.in_stride % (16 / sizeof(TIn)) == 0;
      float2 x[Q][8];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int k = rank * kSlab + int(threadIdx.x) + S::kThreads * q;
        const TIn* src = in + (long long)k * a.in_stride + line0;
        if (seg) {
          Seg8<TIn>::load(src, x[q]);
        } else {
#pragma unroll
          for (int l = 0; l < 8; ++l)
            x[q][l] = line0 + l < a.lines ? Storage<TIn>::load(src + l) : make_float2(0.f, 0.f);
        }
      }
      // Every CTA of the cluster must be running before its shared memory is written.
      cluster_barrier<S>();
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int k = rank * kSlab + int(threadIdx.x) + S::kThreads * q;
#pragma unroll
        for (int l = 0; l < 8; ++l) cluster_store<S>(smem_rows, l, pad16(k), x[q][l]);
      }
    } else {
      float2 x[P];
#pragma unroll
      for (int i = 0; i < P; ++i) {
        const int idx = threadIdx.x + i * S::kThreads;
        const int l = idx % S::kLinesPerCluster;
        const int k = rank * kSlab + idx / S::kLinesPerCluster;
        const long long ln = line0 + l;
        x[i] = ln < a.lines ? Storage<TIn>::load(in + (long long)k * a.in_stride + ln) : make_float2(0.f, 0.f);
      }
      cluster_barrier<S>();
#pragma unroll
      for (int i = 0; i < P; ++i) {
        const int idx = threadIdx.x + i * S::kThreads;
        const int l = idx % S::kLinesPerCluster;
        const int k = rank * kSlab + idx / S::kLinesPerCluster;
        cluster_store<S>(smem_rows, l, pad16(k), x[i]);
      }
    }
    cluster_barrier<S>();
    if constexpr (S::kLinesPerCluster == 8 && std::is_same<TIn, __half2>::value) {
      const uint32_t* sh = reinterpret_cast<const uint32_t*>(sm);
#pragma unroll
      for (int m = 0; m < P; ++m) v[m] = bits_half2(sh[pad16(t + T * m)]);
    } else {
#pragma unroll
      for (int m = 0; m < P; ++m) v[m] = sm[pad16(t + T * m)];
    }
    __syncthreads();
  } else if (active) {
    if (a.pf_ahead > 0) {
      // Dense rows: one bulk L2 prefetch of the lines of the CTA that will
      // take this one's slot about one resident wave later (listed lines:
      // one prefetch per line, by its group's first thread).
      const long long l0 = ((long long)blockIdx.x + a.pf_ahead) * S::G;
      if (a.line_off == nullptr) {
        const long long cnt = a.lines - l0 < S::G ? a.lines - l0 : S::G;
        if (threadIdx.x == 0 && cnt > 0)
          prefetch_l2_bulk(static_cast<const TIn*>(a.in) + l0 * N, uint32_t(cnt * N * sizeof(TIn)));
      } else if (t == 0 && l0 + g < a.lines) {
        prefetch_l2_bulk(static_cast<const TIn*>(a.in) + a.line_off[l0 + g], uint32_t(N * sizeof(TIn)));
      }
    }
    const TIn* in = static_cast<const TIn*>(a.in) + line_start(a, line, a.in_stride) + t;
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = Storage<TIn>::load(in + T * m);
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = make_float2(0.f, 0.f);
  }
  if constexpr (XV == kXchF32) {
    row_compute<N, MODE, NAIVE, SCALED>(v, a, sm, t, line);
  } else {
    unsigned char* base = reinterpret_cast<unsigned char*>(smem_rows) + g * XchSel<N, XV>::kLineBytes;
    row_compute_x<N, MODE, NAIVE, SCALED>(v, a, XchSel<N, XV>::make(base), t, line);
  }

  if constexpr (TSTORE && S::kLinesPerCluster == 8 && std::is_same<TOut, __half2>::value) {
    // FP16 output: the line is staged already rounded to half2 (the one
    // rounding it gets anyway), so the pull moves half the bytes.
    uint32_t* sh = reinterpret_cast<uint32_t*>(sm);
#pragma unroll
    for (int m = 0; m < P; ++m) sh[pad16(t + T * m)] = half2_bits(v[m]);
    cluster_barrier<S>();
    constexpr int Q = kSlab / S::kThreads;   // points per thread (2)
    const bool seg = line0 + 8 <= a.lines && a.out_stride % 4 == 0;
    __half2* out = static_cast<__half2*>(a.out);
    uint32_t w[Q][8];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int k = rank * kSlab + int(threadIdx.x) + S::kThreads * q;
#pragma unroll
      for (int l = 0; l < 8; ++l) {
        const uint32_t* slot = reinterpret_cast<const uint32_t*>(smem_rows + (l % S::G) * S::kSmemPerLine) + pad16(k);
        if constexpr (S::C > 1) {
          w[q][l] = ld_cluster_b32(mapa(smem_addr(slot), uint32_t(l / S::G)));
        } else {
          w[q][l] = *slot;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int k = rank * kSlab + int(threadIdx.x) + S::kThreads * q;
      __half2* dst = out + (long long)k * a.out_stride + line0;
      if (seg) {
        seg8_store_raw(dst, w[q]);
      } else {
#pragma unroll
        for (int l = 0; l < 8; ++l)
          if (line0 + l < a.lines) __stcs(reinterpret_cast<unsigned int*>(dst + l), w[q][l]);
      }
    }
    if constexpr (S::C > 1) {
      cluster_barrier_relaxed();
    } else {
      __syncthreads();
    }
  } else if constexpr (TSTORE) {
    // Stage the line, then every CTA pulls its slab of all cluster lines from
    // the peers' row buffers and writes it as segments.  The last pass read
    // shared memory before a barrier, so the slots are free.  (Pulling with
    // remote loads measured faster than pushing with remote stores, whose
    // release barrier waits for every store to land.)
#pragma unroll
    for (int m = 0; m < P; ++m) sm[pad16(t + T * m)] = v[m];
    cluster_barrier<S>();
    // With 8 lines per cluster a thread owns two points of this CTA's slab:
    // it loads each point's value from the 8 lines (a warp's loads go to one
    // CTA, 32 consecutive points) and writes them as one contiguous 8-line
    // segment of output row k (32 B in FP16).  All loads are in flight before
    // the first store.
    static_assert(kSlab * S::kLinesPerCluster == P * S::kThreads, "one slot per thread and point");
    TOut* out = static_cast<TOut*>(a.out);
    if constexpr (S::kLinesPerCluster == 8) {
      constexpr int Q = kSlab / S::kThreads;   // points per thread (2)
      const bool seg = line0 + 8 <= a.lines && a.out_stride % (16 / sizeof(TOut)) == 0;
      float2 w[Q][8];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int k = rank * kSlab + int(threadIdx.x) + S::kThreads * q;
#pragma unroll
        for (int l = 0; l < 8; ++l) w[q][l] = cluster_load<S>(smem_rows, l, pad16(k));
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int k = rank * kSlab + int(threadIdx.x) + S::kThreads * q;
        TOut* dst = out + (long long)k * a.out_stride + line0;
        if (seg) {
          Seg8<TOut>::store(dst, w[q]);
        } else {
#pragma unroll
          for (int l = 0; l < 8; ++l)
            if (line0 + l < a.lines) Storage<TOut>::store(dst + l, w[q][l]);
        }
      }
    } else {
      float2 w[P];
#pragma unroll
      for (int i = 0; i < P; ++i) {
        const int idx = threadIdx.x + i * S::kThreads;
        const int l = idx % S::kLinesPerCluster;
        const int k = rank * kSlab + idx / S::kLinesPerCluster;
        w[i] = cluster_load<S>(smem_rows, l, pad16(k));
      }
#pragma unroll
      for (int i = 0; i < P; ++i) {
        const int idx = threadIdx.x + i * S::kThreads;
        const int l = idx % S::kLinesPerCluster;
        const int k = rank * kSlab + idx / S::kLinesPerCluster;
        const long long ln = line0 + l;
        if (ln < a.lines) Storage<TOut>::store(out + (long long)k * a.out_stride + ln, w[i]);
      }
    }
    // Keep this CTA's shared memory alive until every peer has read it.  The
    // peers' remote loads have completed once they arrive, so a relaxed
    // barrier suffices (a release barrier would wait for the global stores).
    if constexpr (S::C > 1) {
      cluster_barrier_relaxed();
    } else {
      __syncthreads();
    }
  } else if (active) {
    TOut* out = static_cast<TOut*>(a.out) + line_start(a, line, a.out_stride) + t;
#pragma unroll
    for (int m = 0; m < P; ++m) Storage<TOut>::store(out + T * m, v[m]);
    check_finite<Storage<TOut>, P>(a.finite_flag, [&](int m) { return v[m]; });
  }
}


// Persistent, software-pipelined variant for dense rows (stride == N, no
// corner turn).  Each CTA walks groups of G lines grid-stride; one thread
// keeps STAGES groups in flight with bulk asynchronous copies (TMA) into
// shared-memory stages while the CTA transforms the current group, so HBM
// reads overlap the butterflies.  Stores go straight from registers to HBM
// (coalesced).  Waits are bounded: on expiry the CTA records a timeout in
// a.status, drains its own outstanding copies (again bounded) and returns.
constexpr size_t kTmaSmemBudget = 200 * 1024;   // leave room below the 227 KB per-CTA limit

template <int N, class TIn, int STAGES, int XV = kXchF32>
struct TmaLayout {
  using S = RowShape<N>;
  static constexpr size_t kStageBytes = size_t(S::G) * N * sizeof(TIn);
  static constexpr size_t kBarBytes = 128;
  static constexpr size_t kXchBytes = size_t(S::G) * XchSel<N, XV>::kLineBytes;
  static constexpr size_t kBytes = kBarBytes + STAGES * kStageBytes + kXchBytes;
};

template <int N, class TIn, class TOut, int MODE, bool NAIVE, bool SCALED, int STAGES, int XV = kXchF32>
__global__ void __launch_bounds__(RowShape<N>::kThreads, RowShape<N>::kMinBlocks)
fft_rows_tma_kernel(const RowArgs a) {
  using S = RowShape<N>;
  using L = TmaLayout<N, TIn, STAGES, XV>;
  constexpr int P = S::P, T = S::T, G = S::G;
  extern __shared__ __align__(128) unsigned char smem_tma[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_tma);
  unsigned char* stages = smem_tma + L::kBarBytes;
  unsigned char* xch = stages + STAGES * L::kStageBytes;
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  unsigned char* xg = xch + g * XchSel<N, XV>::kLineBytes;
  const long long groups = (a.lines + G - 1) / G;
  const TIn* src = static_cast<const TIn*>(a.in);

  auto issue = [&](long long grp, int stage) {
    const long long first = grp * G;
    const long long valid = a.lines - first < G ? a.lines - first : G;
    const uint32_t bytes = uint32_t(valid * N * sizeof(TIn));
    mbar_arrive_expect_tx(&bars[stage], bytes);
    bulk_load(stages + stage * L::kStageBytes, src + first * N, bytes, &bars[stage]);
  };

  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
    fence_proxy_async_shared();
#pragma unroll
    for (int s = 0; s < STAGES; ++s) {
      const long long grp = blockIdx.x + (long long)s * gridDim.x;
      if (grp < groups) issue(grp, s);
    }
  }
  __syncthreads();

  int it = 0;
  for (long long grp = blockIdx.x; grp < groups; grp += gridDim.x, ++it) {
    const int stage = it % STAGES;
    const uint32_t parity = (it / STAGES) & 1;
    const bool arrived = mbar_wait_bounded(&bars[stage], parity, a.status);
    float2 v[P];
    const TIn* st = reinterpret_cast<const TIn*>(stages + stage * L::kStageBytes) + g * N + t;
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = Storage<TIn>::load_smem(st + T * m);
    // All threads agree on a timeout; the stage is free once everyone has read it.
    if (__syncthreads_or(!arrived)) {
      if (threadIdx.x == 0) {
        for (int k = 1; k < STAGES; ++k) {             // drain copies still in flight
          const long long later = grp + (long long)k * gridDim.x;
          if (later < groups) mbar_wait_bounded(&bars[(it + k) % STAGES], ((it + k) / STAGES) & 1, nullptr);
        }
      }
      __syncthreads();
      return;
    }
    if (threadIdx.x == 0) {
      const long long nxt = grp + (long long)STAGES * gridDim.x;
      if (nxt < groups) {
        fence_proxy_async_shared();
        issue(nxt, stage);
      }
    }
    int ti;   // opaque per iteration: no address arithmetic carried across the loop
    asm volatile("mov.b32 %0, %1;" : "=r"(ti) : "r"(t));
    const long long line = grp * G + g;
    row_compute_x<N, MODE, NAIVE, SCALED>(v, a, XchSel<N, XV>::make(xg), ti, line);
    if (line < a.lines) {
      TOut* out = static_cast<TOut*>(a.out) + line * a.out_stride + t;
#pragma unroll
      for (int m = 0; m < P; ++m) Storage<TOut>::store(out + T * m, v[m]);
      check_finite<Storage<TOut>, P>(a.finite_flag, [&](int m) { return v[m]; });
    }
  }
}

// One-time host set-up of a kernel: the dynamic shared-memory attribute when
// above 48 KB, and the number of its CTAs resident on the whole device.
// Launchers keep the result in a function-local static, which C++ initialises
// exactly once even when several host threads make the first call together
// (one process per GPU: the device of that first call).
struct LaunchSetup {
  cudaError_t err;
  int resident;
};

template <class K>
LaunchSetup setup_kernel(K kern, int threads, size_t smem) {
  LaunchSetup r{cudaSuccess, 0};
  if (smem > 48 * 1024) {
    r.err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (r.err != cudaSuccess) return r;
  }
  int dev = 0, sms = 0, per_sm = 0;
  if ((r.err = cudaGetDevice(&dev)) != cudaSuccess) return r;
  if ((r.err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return r;
  if ((r.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem)) != cudaSuccess) return r;
  r.resident = (per_sm > 0 ? per_sm : 1) * sms;
  return r;
}

template <int N, class TIn, class TOut, int MODE, bool NAIVE, bool SCALED, int XV = kXchF32>
cudaError_t launch_rows_tma_n(const RowArgs& a, cudaStream_t stream) {
  using S = RowShape<N>;
  constexpr int kStages = 2;
  using L = TmaLayout<N, TIn, kStages, XV>;
  auto kern = fft_rows_tma_kernel<N, TIn, TOut, MODE, NAIVE, SCALED, kStages, XV>;
  static const LaunchSetup setup = setup_kernel(kern, S::kThreads, L::kBytes);
  if (setup.err != cudaSuccess) return setup.err;
  const int grid_cap = setup.resident;
  if (a.lines <= 0) return cudaSuccess;
  const long long groups = (a.lines + S::G - 1) / S::G;
  const int grid = int(groups < grid_cap ? groups : grid_cap);
  kern<<<dim3(grid), dim3(S::kThreads), L::kBytes, stream>>>(a);
  return cudaGetLastError();
}



// Four-step line of N = N1 * 4096 points over a group of N1 CTAs (N1 = 2, 4,
// 8, 16) of one thread-block cluster, 256 threads each.  With n = n2 + 4096 n1
// and k = k1 + N1 k2:
//   X[k1 + N1 k2] = sum_n2 W_4096^{n2 k2} W_N^{n2 k1} sum_n1 x[n2 + 4096 n1] W_N1^{n1 k1}.
// Step 1: CTA c loads the n2-slab [c S, (c + 1) S) (S = 4096 / N1) of every
//   block n1 -- N1 contiguous, coalesced segments -- runs the N1-point DFTs in
//   registers, multiplies by W_N^{n2 k1} and sends row k1 to CTA k1's shared
//   memory with asynchronous remote stores (st.async) that count their bytes
//   on CTA k1's mbarrier: the one exchange through distributed shared memory,
//   with no cluster barrier (whose release would wait for global stores).
// Step 2: CTA k1 transforms its row (4096 points, local Stockham passes).
// Step 3 (N1 >= 8): natural-order output, 4096 contiguous points per CTA: CTA
//   k1 sends X[k1 + N1 k2] to the output buffer of CTA k2 / S with st.async
//   counted on that CTA's second mbarrier (a warp's 32 values go to one CTA,
//   contiguous; FP16 storage sends the rounded half2 words, the one rounding
//   the store makes anyway), waits for its own 4096 points and writes them
//   with coalesced stores.  For N1 = 16 storing X[k1 + N1 k2] straight from
//   step 2 scatters every warp store over 32 sectors (35-40 % slower); for
//   N1 <= 4 the direct strided store is faster than the exchange, which makes
//   each CTA wait for its whole group.
// Both exchanges only wait on data, never on a cluster barrier.  A CTA's row
// buffer is free again once it has sent its step-3 values, and its output
// buffer once it has stored them; no peer can send into either for the next
// line before receiving this CTA's contributions to that line, so lines on
// the same CTAs need no barrier in between.
// The caller provides `smem` with a row buffer of pad16(4096) points followed
// by the output buffer (fourstep_smem_bytes in all), initialises `bar` and
// `bar_out` (one arrival each) and makes them visible to the cluster before
// the first line.
// Expired waits.  Both receive waits are bounded (mbar_wait_bounded); the
// threads of the CTA agree on an expiry with __syncthreads_or, and the line
// then returns false at once, with `pending` naming the receive barriers whose
// phase `phase` has not completed (bit 0: row, bit 1: output).  The caller
// must then stop sending and waiting (no further line on these barriers) and,
// before the CTA exits, call fourstep_drain so that peers' stores still in
// flight land before its shared memory goes away.
// The FP8 pair (satfinite RN) of v as the low 16 bits of a word.
template <class TS>
__device__ __forceinline__ uint32_t fp8_pair_bits(float2 v) {
  return uint32_t(__nv_cvt_float2_to_fp8x2(v, __NV_SATFINITE, Fp8Format<TS>::kInterp));
}

// Step-3 send words: FP32 pairs; for FP16 storage the rounded half2; for FP8
// storage two rounded FP8 pairs, those of consecutive k2 (the values are
// rounded where they are computed, as the owner would round them).  In the
// owner's buffer, segment k1 holds word w at w ^ (k1 * kSwz(N1)): a warp's
// sends stay one aligned block (the XOR stays below 32) and the owner's
// gather, which reads the same w of up to 16 segments at once, spreads over
// distinct banks (16 lanes a wavefront for 8-byte words, 32 for 4-byte).
template <class TS> struct FsSend {
  using Word = float2;
  static constexpr int kPts = 1;
  __host__ __device__ static constexpr int swz(int n1) { return 16 / n1; }
};
template <> struct FsSend<__half2> {
  using Word = uint32_t;
  static constexpr int kPts = 1;
  __host__ __device__ static constexpr int swz(int n1) { return 32 / n1; }
};
template <class F> struct FsSend<Fp8x2<F>> {
  using Word = uint32_t;
  static constexpr int kPts = 2;
  __host__ __device__ static constexpr int swz(int n1) { return 32 / n1; }
};
// Shared memory of a four-step line: the row buffer, and for N1 >= 8 the
// output buffer of N1 segments of S / kPts words, S = 4096 / N1.
template <class TS, int N1>
__host__ __device__ constexpr size_t fourstep_smem_bytes() {
  using X = FsSend<TS>;
  return size_t(pad16(4096)) * sizeof(float2) +
         (N1 >= 8 ? size_t(4096 / X::kPts) * sizeof(typename X::Word) : 0);
}

template <int N1, class TS, int MODE, bool SCALED, bool H16ROW = false>
__device__ __forceinline__ bool fourstep_line(const RowArgs& a, const TS* in, TS* out, float2* smem, uint64_t* bar,
                                              uint64_t* bar_out, uint32_t& phase, int& pending, int c,
                                              int base_rank, bool active) {
  constexpr int N = N1 * 4096, S = 4096 / N1, NB = 16 / N1, P = kPointsPerThread;
  const int t = threadIdx.x;
  const float inv_n = 1.0f / float(N);
  // This CTA receives its row and its output range: 4096 points of 8 bytes
  // each, from all N1 CTAs.
  constexpr bool kOutXch = N1 >= 8;
  using Word = typename FsSend<TS>::Word;
  constexpr int kPts = FsSend<TS>::kPts;                // points per send word
  constexpr int kSeg = S / kPts;                        // words per segment of the owner's buffer
  constexpr int kSwz = FsSend<TS>::swz(N1);
  static_assert(!kOutXch || (kSwz * (N1 - 1) < 32 && kSwz * (N1 - 1) < kSeg), "swizzle within a block");
  // H16ROW with FP16 storage: the row arrives as FP16 words (one more FP16
  // storage point, half the exchange bytes); otherwise as FP32 pairs.
  constexpr bool h16row = H16ROW && std::is_same<TS, __half2>::value;
  if (t == 0) {
    mbar_arrive_expect_tx(bar, 4096u * uint32_t(h16row ? sizeof(uint32_t) : sizeof(float2)));
    if constexpr (kOutXch) mbar_arrive_expect_tx(bar_out, uint32_t(4096 / kPts * sizeof(Word)));
  }
  float2* smem_out = smem + pad16(4096);
  const uint32_t smem_base = smem_addr(smem), bar_local = smem_addr(bar);
  const uint32_t out_base = smem_addr(smem_out), bar_out_local = smem_addr(bar_out);
  float2 v[P];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int n2 = c * S + t + 256 * b;
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1)
      v[b * N1 + n1] = active ? Storage<TS>::load(in + n2 + 4096 * n1) : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int m = 0; m < P; ++m) {
    if (SCALED) v[m] = cscale(v[m], a.in_scale);
    if (MODE == kInverse) v[m] = cscale(cconj(v[m]), inv_n);
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int n2 = c * S + t + 256 * b;
    float2 u[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) u[i] = v[b * N1 + i];
    Dft<N1>::run(u);
    const uint32_t slot = h16row ? smem_base + uint32_t(n2) * 4u : smem_base + uint32_t(n2) * uint32_t(sizeof(float2));
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const float2 z = k1 == 0 ? u[0] : cmul(u[k1], __ldg(a.tw_4step + k1 * 4096 + n2));
      if constexpr (h16row) {
        st_async_b32(mapa(slot, base_rank + k1), half2_bits(z), mapa(bar_local, base_rank + k1));
      } else {
        st_async_f2(mapa(slot, base_rank + k1), z, mapa(bar_local, base_rank + k1));
      }
    }
  }
  // The row is complete when all of it has landed (bounded wait).  It sits
  // unpadded at n2: each warp's sends then fill aligned 128- or 256-byte
  // segments of the owner's buffer (padded slots measured 8-10 % slower),
  // and the reads below are conflict-free without padding.
  const bool row_ok = mbar_wait_bounded(bar, phase, a.status);
#pragma unroll
  for (int m = 0; m < P; ++m)
    v[m] = h16row ? bits_half2(reinterpret_cast<const uint32_t*>(smem)[t + 256 * m]) : smem[t + 256 * m];
  if (__syncthreads_or(!row_ok)) {
    pending = kOutXch ? 3 : 1;
    return false;
  }
  line_dft<4096>(v, a.tw_line, smem, t);
#pragma unroll
  for (int m = 0; m < P; ++m) {
    if (MODE == kInverse) v[m] = cconj(v[m]);
    if (SCALED) v[m] = cscale(v[m], a.out_scale);
  }
  if constexpr (!kOutXch) {
    phase ^= 1;
    if (active) {
#pragma unroll
      for (int m = 0; m < P; ++m) Storage<TS>::store(out + c + N1 * (t + 256 * m), v[m]);
      check_finite<Storage<TS>, P>(a.finite_flag, [&](int m) { return v[m]; });
    }
    return true;
  } else {
    // The owner's buffer holds the values as [k1][k2 mod S] in segments of
    // kSeg words (swizzled, see FsSend), so a warp's sends fill one aligned
    // block; the owner gathers output position j = (k2 mod S) N1 + k1 from
    // segment k1, point j / N1.  FP8
    // words hold the points of k2 and k2 + 1 (k2 even): for even m the even
    // thread of each lane pair sends its value and its odd partner's, for odd
    // m the odd thread does.
#pragma unroll
    for (int m = 0; m < P; ++m) {
      const int k2 = t + 256 * m;
      const uint32_t dst = uint32_t(base_rank + k2 / S);
      if constexpr (kPts == 2) {
        const uint32_t own = fp8_pair_bits<TS>(v[m]);
        const uint32_t other = __shfl_xor_sync(0xffffffffu, own, 1);
        if ((t & 1) == (m & 1)) {
          const uint32_t w = t & 1 ? other | (own << 16) : own | (other << 16);
          const uint32_t slot = out_base + uint32_t(c * kSeg + (((k2 % S) / 2) ^ (kSwz * c))) * uint32_t(sizeof(Word));
          st_async_b32(mapa(slot, dst), w, mapa(bar_out_local, dst));
        }
      } else {
        const uint32_t slot = out_base + uint32_t(c * kSeg + ((k2 % S) ^ (kSwz * c))) * uint32_t(sizeof(Word));
        if constexpr (sizeof(Word) == 4) {
          st_async_b32(mapa(slot, dst), half2_bits(v[m]), mapa(bar_out_local, dst));
        } else {
          st_async_f2(mapa(slot, dst), v[m], mapa(bar_out_local, dst));
        }
      }
    }
    const bool out_ok = mbar_wait_bounded(bar_out, phase, a.status);
    if (__syncthreads_or(!out_ok)) {
      pending = 2;
      return false;
    }
    phase ^= 1;
    if (active) {
      const Word* ob = reinterpret_cast<const Word*>(smem_out);
      if constexpr (kPts == 2) {
        auto bits = [&](int m) -> uint16_t {
          const int j = t + 256 * m, q = j / N1;
          return uint16_t(ob[(j % N1) * kSeg + ((q / 2) ^ (kSwz * (j % N1)))] >> (16 * (q & 1)));
        };
#pragma unroll
        for (int m = 0; m < P; ++m)
          __stcs(reinterpret_cast<unsigned short*>(out + c * 4096 + t + 256 * m), bits(m));
        check_finite<Storage<TS>, P>(a.finite_flag, [&](int m) {
          TS pair;
          pair.bits = bits(m);
          return Storage<TS>::load_smem(&pair);
        });
      } else {
#pragma unroll
        for (int m = 0; m < P; ++m) {
          const int j = t + 256 * m;
          const Word w = ob[(j % N1) * kSeg + ((j / N1) ^ (kSwz * (j % N1)))];
          if constexpr (sizeof(Word) == 4) {
            __stcs(reinterpret_cast<unsigned int*>(out + c * 4096 + j), w);
          } else {
            Storage<TS>::store(out + c * 4096 + j, w);
          }
        }
        if constexpr (sizeof(Word) == 4) {
          check_finite<Storage<TS>, P>(a.finite_flag, [&](int m) {
            const int j = t + 256 * m;
            return bits_half2(ob[(j % N1) * kSeg + ((j / N1) ^ (kSwz * (j % N1)))]);
          });
        } else {
          check_finite<Storage<TS>, P>(a.finite_flag, [&](int m) {
            const int j = t + 256 * m;
            return ob[(j % N1) * kSeg + ((j / N1) ^ (kSwz * (j % N1)))];
          });
        }
      }
    }
    return true;
  }
}

// After a fourstep_line that returned false: wait (bounded, once more) for the
// pending receive phases, so that no peer's asynchronous store still targets
// this CTA's shared memory when it exits.  Peers send into this CTA only what
// the line's protocol owes it, so these phases complete unless a peer stopped
// sending; then nothing is in flight and the wait simply expires.
__device__ __forceinline__ void fourstep_drain(uint64_t* bar, uint64_t* bar_out, uint32_t phase, int pending) {
  if (pending & 1) mbar_wait_bounded(bar, phase, nullptr);
  if (pending & 2) mbar_wait_bounded(bar_out, phase, nullptr);
  __syncthreads();
}

// Uniform plans with N >= 8192: one line per group of N / 4096 CTAs, a
// cluster per line.
template <int N, class TS, int MODE, bool SCALED, bool H16ROW>
// Four CTAs per SM (64 registers) where their shared memory fits, else three.
__global__ void __launch_bounds__(256, fourstep_smem_bytes<TS, N / 4096>() * 4 <= 220 * 1024 ? 4 : 3)
    fft_fourstep_kernel(const RowArgs a) {
  constexpr int N1 = N / 4096;
  extern __shared__ float2 smem_fs[];
  __shared__ __align__(8) uint64_t bar, bar_out;
  auto cluster = cooperative_groups::this_cluster();
  const int c = int(cluster.block_rank());
  const long long line = blockIdx.x / N1;
  const TS* in = static_cast<const TS*>(a.in) + line_start(a, line, a.in_stride);
  TS* out = static_cast<TS*>(a.out) + line_start(a, line, a.out_stride);
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init(&bar_out, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // Dense lines: prefetch this CTA's share of the line one resident wave
    // of clusters later into L2.
    if (a.pf_ahead > 0 && line + a.pf_ahead < a.lines)
      prefetch_l2_bulk(static_cast<const TS*>(a.in) + line_start(a, line + a.pf_ahead, N) + c * 4096,
                       uint32_t(4096 * sizeof(TS)));
  }
  // Every CTA running, every mbarrier initialised: the initialisation is
  // published by its own release fence, so the arrive can be relaxed (no
  // memory barrier for the other threads).
  cluster_arrive_relaxed();
  cluster_wait_acquire();
  uint32_t phase = 0;
  int pending = 0;
  if (!fourstep_line<N1, TS, MODE, SCALED, H16ROW>(a, in, out, smem_fs, &bar, &bar_out, phase, pending, c, 0, true))
    fourstep_drain(&bar, &bar_out, phase, pending);
  // No CTA leaves while a peer's asynchronous stores may still be in flight:
  // every CTA has received what it waited for (or drained it) before arriving.
  cluster_barrier_relaxed();
}

template <int N, class TS, int MODE, bool SCALED, bool H16ROW = false>
cudaError_t launch_fourstep_n(const RowArgs& a, cudaStream_t stream) {
  constexpr int N1 = N / 4096;
  constexpr size_t kBytes = fourstep_smem_bytes<TS, N / 4096>();
  auto kern = fft_fourstep_kernel<N, TS, MODE, SCALED, H16ROW>;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = kBytes;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = N1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // One-time set-up (thread-safe, see setup_kernel): attributes and the
  // number of resident clusters.
  static const LaunchSetup setup = [&]() -> LaunchSetup {
    LaunchSetup r{cudaSuccess, 0};
    if (N1 > 8) {
      r.err = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (r.err != cudaSuccess) return r;
    }
    r.err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kBytes));
    if (r.err != cudaSuccess) return r;
    cudaLaunchConfig_t probe = cfg;
    probe.gridDim = dim3(N1);
    r.err = cudaOccupancyMaxActiveClusters(&r.resident, kern, &probe);
    return r;
  }();
  if (setup.err != cudaSuccess) return setup.err;
  const int resident_clusters = setup.resident;
  if (a.lines <= 0) return cudaSuccess;
  const long long grid = a.lines * N1;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  cfg.gridDim = dim3(unsigned(grid));
  RowArgs b = a;
  b.pf_ahead = (a.variant == kRowsPlainL2 || a.variant == kRowsPlain4L2 || a.variant == kRowsPlainHL2 ||
                a.variant == kRowsPlainH4L2 || a.variant == kRowsPlainHS4L2)
                   ? resident_clusters
                   : 0;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, b);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// Lines longer than one CTA's share (N >= 8192): a line spans a thread-block
// cluster of C CTAs of CTA_T threads, each CTA holding a slab of N / C points
// of every exchange in its shared memory; the passes read and write the other
// CTAs' slabs through distributed shared memory and synchronise with cluster
// barriers.  Each line is still read from and written to HBM exactly once.
template <int N>
struct ClusterShape {
  static constexpr int CTA_T = N <= 32768 ? 256 : 512;
  static constexpr int T = N / kPointsPerThread;   // threads per line
  static constexpr int C = T / CTA_T;              // CTAs per line (cluster size, <= 8)
  static constexpr int SLAB = N / C;               // points per CTA
  static constexpr size_t kSmemBytes = size_t(pad16(SLAB)) * sizeof(float2);
  static constexpr int kMinBlocks = CTA_T >= 512 ? 1 : BFP_MIN_BLOCKS;
  static_assert(C >= 2 && C <= 8, "cluster size");
};

template <int N, class TIn, class TOut, int MODE, bool NAIVE, bool SCALED>
__global__ void __launch_bounds__(ClusterShape<N>::CTA_T, ClusterShape<N>::kMinBlocks)
fft_cluster_kernel(const RowArgs a) {
  using S = ClusterShape<N>;
  constexpr int P = kPointsPerThread, T = S::T;
  extern __shared__ float2 smem_cl[];
  auto cluster = cooperative_groups::this_cluster();
  const int rank = int(cluster.block_rank());
  const long long line = blockIdx.x / S::C;
  const int t = rank * S::CTA_T + threadIdx.x;
  const ClusterXch<S::SLAB> xch{smem_cl};
  float2 v[P];
  const TIn* in = static_cast<const TIn*>(a.in) + line * a.in_stride + t;
#pragma unroll
  for (int m = 0; m < P; ++m) v[m] = Storage<TIn>::load(in + T * m);
  // Every CTA of the cluster must be running before its slab is written.
  cluster.sync();
  row_compute_x<N, MODE, NAIVE, SCALED>(v, a, xch, t, line);
  // The last exchange ended with a cluster barrier after its reads: no CTA
  // touches another's slab from here on.
  TOut* out = static_cast<TOut*>(a.out) + line * a.out_stride + t;
#pragma unroll
  for (int m = 0; m < P; ++m) Storage<TOut>::store(out + T * m, v[m]);
  check_finite<Storage<TOut>, P>(a.finite_flag, [&](int m) { return v[m]; });
}

template <int N, class TIn, class TOut, int MODE, bool NAIVE, bool SCALED>
cudaError_t launch_cluster_n(const RowArgs& a, cudaStream_t stream) {
  using S = ClusterShape<N>;
  auto kern = fft_cluster_kernel<N, TIn, TOut, MODE, NAIVE, SCALED>;
  static const LaunchSetup setup = setup_kernel(kern, S::CTA_T, S::kSmemBytes);
  if (setup.err != cudaSuccess) return setup.err;
  if (a.lines <= 0) return cudaSuccess;
  const long long grid = a.lines * S::C;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(S::CTA_T);
  cfg.dynamicSmemBytes = S::kSmemBytes;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = S::C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// Tensor-core radix-16 variant (tc_fft.cuh), N = 4096, FP16 storage.
template <class TS, int MODE>
cudaError_t launch_tc_n(const RowArgs& a, cudaStream_t stream);

// Plain row kernel (one group per CTA) with an exchange variant; optionally
// each CTA prefetches into L2 the lines of the CTA one resident wave later.
template <int N, class TIn, class TOut, int MODE, bool NAIVE, int XV, int MINB = 0>
cudaError_t launch_rows_plain_x(const RowArgs& a, cudaStream_t stream, bool l2_prefetch = false) {
  using S = RowShape<N>;
  constexpr size_t kBytes = size_t(S::G) * XchSel<N, XV>::kLineBytes;
  auto kern = fft_rows_kernel<N, TIn, TOut, MODE, NAIVE, false, false, false, XV, MINB>;
  static const LaunchSetup setup = setup_kernel(kern, S::kThreads, kBytes);
  if (setup.err != cudaSuccess) return setup.err;
  const int resident = setup.resident;   // CTAs of this kernel resident on the whole GPU
  if (a.lines <= 0) return cudaSuccess;
  const long long grid = (a.lines + S::G - 1) / S::G;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  RowArgs b = a;
  b.pf_ahead = l2_prefetch ? resident : 0;
  kern<<<dim3(unsigned(grid)), dim3(S::kThreads), kBytes, stream>>>(b);
  return cudaGetLastError();
}

template <int N, class TIn, class TOut, int MODE, bool NAIVE, bool SCALED, bool TLOAD = false,
          bool TSTORE = false>
cudaError_t launch_rows_n(const RowArgs& a, cudaStream_t stream) {
  // Dense lines of 32768 and 65536 points: the four-step kernel over a
  // cluster.  Lines of 8192 and 16384 points run on one CTA of N / 16 threads
  // (512 at 2 CTAs per SM, or 1024), which measured 1.4x faster than the
  // four-step kernel for plain transforms and 3x faster than the per-pass
  // cluster kernel for compression; longer lines the four-step kernel does not
  // take (compression, naive FP16, mixed storage, strided rows) need the
  // cluster kernel.
  if constexpr (!TLOAD && !TSTORE && N >= 32768) {
    if constexpr (MODE != kCompress && !NAIVE && std::is_same<TIn, TOut>::value) {
      if (a.tw_4step != nullptr && a.in_stride == N && a.out_stride == N) {
        if constexpr (std::is_same<TIn, __half2>::value) {
          if (a.fs_h16) return launch_fourstep_n<N, TIn, MODE, SCALED, true>(a, stream);
        }
        return launch_fourstep_n<N, TIn, MODE, SCALED>(a, stream);
      }
    }
  }
  if constexpr (!TLOAD && !TSTORE && N > 16384) {
    return launch_cluster_n<N, TIn, TOut, MODE, NAIVE, SCALED>(a, stream);
  } else {
  using S = RowShape<N, TLOAD || TSTORE>;
  // Exchange variants for dense forward / inverse rows (FP16 exchange only
  // for FP16 storage): see RowVariant.
  if constexpr (!TLOAD && !TSTORE && !SCALED && MODE != kCompress && N >= 256 && N <= 4096 &&
                std::is_same<TIn, TOut>::value) {
    if (a.in_stride == N && a.out_stride == N) {
      constexpr bool kHalf = std::is_same<TIn, __half2>::value;
      switch (a.variant) {
        case kRowsPlainPP: return launch_rows_plain_x<N, TIn, TOut, MODE, NAIVE, kXchF32PP>(a, stream);
        case kRowsPlain4: return launch_rows_plain_x<N, TIn, TOut, MODE, NAIVE, kXchF32, 4>(a, stream);
        case kRowsPlainL2: return launch_rows_plain_x<N, TIn, TOut, MODE, NAIVE, kXchF32>(a, stream, true);
        case kRowsPlain4L2: return launch_rows_plain_x<N, TIn, TOut, MODE, NAIVE, kXchF32, 4>(a, stream, true);
        case kRowsTmaPP: return launch_rows_tma_n<N, TIn, TOut, MODE, NAIVE, SCALED, kXchF32PP>(a, stream);
        case kRowsPlainH:
          if constexpr (kHalf) return launch_rows_plain_x<N, TIn, TOut, MODE, NAIVE, kXchF16>(a, stream);
          break;
        case kRowsPlainHL2:
          if constexpr (kHalf) return launch_rows_plain_x<N, TIn, TOut, MODE, NAIVE, kXchF16>(a, stream, true);
          break;
        case kRowsPlainH4L2:
          if constexpr (kHalf) return launch_rows_plain_x<N, TIn, TOut, MODE, NAIVE, kXchF16, 4>(a, stream, true);
          break;
        case kRowsPlainHS4L2:
          if constexpr (kHalf) return launch_rows_plain_x<N, TIn, TOut, MODE, NAIVE, kXchF16S, 4>(a, stream, true);
          break;
        case kRowsPlainHPP:
          if constexpr (kHalf) return launch_rows_plain_x<N, TIn, TOut, MODE, NAIVE, kXchF16PP>(a, stream);
          break;
        case kRowsTmaH:
          if constexpr (kHalf) return launch_rows_tma_n<N, TIn, TOut, MODE, NAIVE, SCALED, kXchF16>(a, stream);
          break;
        case kRowsTmaHPP:
          if constexpr (kHalf) return launch_rows_tma_n<N, TIn, TOut, MODE, NAIVE, SCALED, kXchF16PP>(a, stream);
          break;
        case kRowsTc:
          if constexpr (kHalf && N == 4096 && !NAIVE) {
            if (a.tc_b != nullptr) return launch_tc_n<TIn, MODE>(a, stream);
          }
          break;
        default: break;
      }
    }
  }
  // Shapes the switch does not cover (scaled FP8 storage, compress mode,
  // mixed storage, corner turns, strided rows) run the pipelined kernel for
  // the TMA family and the generic kernel otherwise.
  const bool tma_family =
      a.variant == kRowsTma || a.variant == kRowsTmaPP || a.variant == kRowsTmaH || a.variant == kRowsTmaHPP;
  if constexpr (!TLOAD && !TSTORE && N >= 256 && TmaLayout<N, TIn, 2>::kBytes <= kTmaSmemBudget) {
    if (tma_family && a.in_stride == N && a.out_stride == N)
      return launch_rows_tma_n<N, TIn, TOut, MODE, NAIVE, SCALED>(a, stream);
  }
  auto kern = fft_rows_kernel<N, TIn, TOut, MODE, NAIVE, SCALED, TLOAD, TSTORE>;
  constexpr size_t kBytes = S::kSmemBytes;
  static const LaunchSetup setup = setup_kernel(kern, S::kThreads, kBytes);
  if (setup.err != cudaSuccess) return setup.err;
  const int resident = setup.resident;   // CTAs of this kernel resident on the whole GPU
  if (a.lines <= 0) return cudaSuccess;
  const long long clusters = (a.lines + S::kLinesPerCluster - 1) / S::kLinesPerCluster;
  const long long grid = clusters * S::C;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  RowArgs b = a;
  const bool l2 = a.variant == kRowsPlainL2 || a.variant == kRowsPlain4L2 || a.variant == kRowsPlainHL2 ||
                  a.variant == kRowsPlainH4L2 || a.variant == kRowsPlainHS4L2;
  b.pf_ahead = (l2 && !TLOAD && a.in_stride == N) ? resident : 0;
  if constexpr (S::C > 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(S::kThreads);
    cfg.dynamicSmemBytes = kBytes;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = S::C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, b);
    if (e != cudaSuccess) return e;
  } else {
    kern<<<dim3(unsigned(grid)), dim3(S::kThreads), kBytes, stream>>>(b);
  }
  return cudaGetLastError();
  }
}

// Dispatch on log2 N in [4, 16] (N >= 32768 only for dense rows).
template <class TIn, class TOut, int MODE, bool NAIVE, bool SCALED, bool TLOAD = false, bool TSTORE = false>
cudaError_t launch_rows(int log2n, const RowArgs& a, cudaStream_t stream) {
  switch (log2n) {
    case 4: return launch_rows_n<16, TIn, TOut, MODE, NAIVE, SCALED, TLOAD, TSTORE>(a, stream);
    case 5: return launch_rows_n<32, TIn, TOut, MODE, NAIVE, SCALED, TLOAD, TSTORE>(a, stream);
    case 6: return launch_rows_n<64, TIn, TOut, MODE, NAIVE, SCALED, TLOAD, TSTORE>(a, stream);
    case 7: return launch_rows_n<128, TIn, TOut, MODE, NAIVE, SCALED, TLOAD, TSTORE>(a, stream);
    case 8: return launch_rows_n<256, TIn, TOut, MODE, NAIVE, SCALED, TLOAD, TSTORE>(a, stream);
    case 9: return launch_rows_n<512, TIn, TOut, MODE, NAIVE, SCALED, TLOAD, TSTORE>(a, stream);
    case 10: return launch_rows_n<1024, TIn, TOut, MODE, NAIVE, SCALED, TLOAD, TSTORE>(a, stream);
    case 11: return launch_rows_n<2048, TIn, TOut, MODE, NAIVE, SCALED, TLOAD, TSTORE>(a, stream);
    case 12: return launch_rows_n<4096, TIn, TOut, MODE, NAIVE, SCALED, TLOAD, TSTORE>(a, stream);
    case 13: return launch_rows_n<8192, TIn, TOut, MODE, NAIVE, SCALED, TLOAD, TSTORE>(a, stream);
    case 14: return launch_rows_n<16384, TIn, TOut, MODE, NAIVE, SCALED, TLOAD, TSTORE>(a, stream);
    case 15:
      if constexpr (!TLOAD && !TSTORE) return launch_rows_n<32768, TIn, TOut, MODE, NAIVE, SCALED>(a, stream);
      else return cudaErrorInvalidValue;
    case 16:
      if constexpr (!TLOAD && !TSTORE) return launch_rows_n<65536, TIn, TOut, MODE, NAIVE, SCALED>(a, stream);
      else return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bfp
