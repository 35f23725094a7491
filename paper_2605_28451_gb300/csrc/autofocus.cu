// Entropy phase autofocus: the image entropy of the azimuth-compressed image
// under a per-pulse phase correction, and its gradient by a hand-written
// adjoint that recomputes the forward transforms instead of storing them.
//
// Model (the paper has no autofocus section; this is standard SAR entropy
// autofocus on top of its azimuth compression, Fig. 1):
//   v[r][n] = rc[r][n] exp(-j phi[n])          rc rows: range bin r, pulse n
//   I[r]    = A v[r],  A = IDFT(DFT(.) . Ha)   azimuth compression of one range bin
//   q = |I|^2,  S = sum q,  p = q / S,  E = -sum p ln p = ln S - (1/S) sum q ln q
// Adjoint:
//   G = dE/dI* = -(ln p + E) / S * I           (0 where q = 0)
//   A^H = IDFT(DFT(.) . conj(Ha))              the same chain with the conjugate filter
//   dE/dphi[n] = 2 sum_r Im( conj((A^H G)[r][n]) * v[r][n] )
//
// Kernels (persistent, one group of N/16 threads per range bin, lines held on
// chip exactly as in fft_rows.cuh):
//   af_phase_kernel     e^{-j phi[n]} table
//   af_kernel<fwd>      per-CTA FP64 partials of S and sum q ln q
//   af_stats_kernel     S, Q, E, ln S (one block, FP64 tree over the partials)
//   af_kernel<bwd>      per-CTA partial gradients (registers across rows)
//   af_grad_kernel      sum of the partial gradients in FP64 (8 slices per 32 pulses)
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "autofocus.h"
#include "fft_rows.cuh"

namespace bfp {

namespace {

struct AfArgs {
  const void* rc;
  const float2* ph;      // e^{-j phi[n]}
  const float2* ha;
  const float2* tw;
  long long rows;        // n_rg
  double* stats;         // S, Q, E, ln S
  double* sq_part;       // [grid][2]
  float* g_part;         // [grid][n_az]
  bool prefetch;         // rc in device memory: prefetch each CTA's next rows into L2
};

__global__ void af_phase_kernel(const float* __restrict__ phi, float2* __restrict__ ph, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    float s, c;
    sincosf(phi[i], &s, &c);
    ph[i] = make_float2(c, -s);
  }
}

// One compression of the line held in v with filter h (conjugated if CONJ_H):
// v <- conj(DFT(conj(DFT(v) . h) / N)).
template <int N, bool CONJ_H>
__device__ __forceinline__ void af_compress(float2 (&v)[kPointsPerThread], const float2* __restrict__ h,
                                            const float2* __restrict__ tw, float2* sm, int t) {
  constexpr int P = kPointsPerThread, T = N / P;
  const float inv_n = 1.0f / float(N);
  // Fresh opaque copies of t for each transform: the compiler must not keep
  // one transform's shared-memory and twiddle addresses live for the next.
  int t1;
  asm volatile("mov.b32 %0, %1;" : "=r"(t1) : "r"(t));
  line_dft<N>(v, tw, sm, t1);
  // Filter loads in groups of four, so the compiler does not hoist all
  // sixteen next to the line (register pressure at 3 CTAs / SM).
#pragma unroll
  for (int m0 = 0; m0 < P; m0 += 4) {
    float2 hv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) hv[i] = __ldg(h + t + T * (m0 + i));
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = CONJ_H ? cconj(hv[i]) : hv[i];
      v[m0 + i] = cscale(cconj(cmul(v[m0 + i], f)), inv_n);
    }
    asm volatile("" ::: "memory");
  }
  int t2;
  asm volatile("mov.b32 %0, %1;" : "=r"(t2) : "r"(t));
  line_dft<N>(v, tw, sm, t2);
#pragma unroll
  for (int m = 0; m < P; ++m) v[m] = cconj(v[m]);
}

// Cached loads (not streaming): the backward kernel reads each row twice and
// the second read should come from L2.
__device__ __forceinline__ float2 load_cached(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float2 load_cached(const __half2* p) {
  const unsigned int u = __ldg(reinterpret_cast<const unsigned int*>(p));
  return __half22float2(*reinterpret_cast<const __half2*>(&u));
}

template <int N, class TIn>
__device__ __forceinline__ void af_load(float2 (&v)[kPointsPerThread], const AfArgs& a, long long row, int t,
                                        bool active) {
  constexpr int P = kPointsPerThread, T = N / P;
  const TIn* in = static_cast<const TIn*>(a.rc) + row * N + t;
  // The line first, then its phases four at a time.
#pragma unroll
  for (int m = 0; m < P; ++m) v[m] = active ? load_cached(in + T * m) : make_float2(0.f, 0.f);
#pragma unroll
  for (int m0 = 0; m0 < P; m0 += 4) {
    float2 p[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) p[i] = __ldg(a.ph + t + T * (m0 + i));
#pragma unroll
    for (int i = 0; i < 4; ++i) v[m0 + i] = cmul(v[m0 + i], p[i]);
    asm volatile("" ::: "memory");
  }
}

// Shared memory of af_kernel: the row buffers, and for the gradient pass one
// FP32 partial gradient per pulse for each line group of the CTA (a thread
// owns the pulses t + T m of its group's slice, so no atomics are needed).
template <int N, bool BACKWARD>
constexpr size_t af_smem_bytes() {
  using S = RowShape<N>;
  return S::kSmemBytes + (BACKWARD ? size_t(S::G) * N * sizeof(float) : 0);
}

template <int N, class TIn, bool BACKWARD>
__global__ void __launch_bounds__(RowShape<N>::kThreads, RowShape<N>::kThreads >= 512 ? 1 : 2)
af_kernel(const AfArgs a) {
  using S = RowShape<N>;
  constexpr int P = S::P, T = S::T, G = S::G;
  extern __shared__ float2 smem_af[];
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  float2* sm = smem_af + g * S::kSmemPerLine;
  float* gsm = reinterpret_cast<float*>(smem_af + G * S::kSmemPerLine) + g * N;   // this group's gradients
  const long long groups = (a.rows + G - 1) / G;

  float s_acc = 0.f, q_acc = 0.f;
  if (BACKWARD) {
#pragma unroll
    for (int m = 0; m < P; ++m) gsm[t + T * m] = 0.f;
  }
  float ln_s_minus_e = 0.f, inv_s = 0.f;
  if (BACKWARD) {
    ln_s_minus_e = float(a.stats[3] - a.stats[2]);   // ln S - E
    inv_s = float(1.0 / a.stats[0]);
  }

  for (long long grp = blockIdx.x; grp < groups; grp += gridDim.x) {
    if (a.prefetch && threadIdx.x == 0 && grp + gridDim.x < groups) {
      // The rows of this CTA's next group, into L2.
      const long long r0 = (grp + gridDim.x) * G;
      const long long cnt = a.rows - r0 < G ? a.rows - r0 : G;
      prefetch_l2_bulk(static_cast<const TIn*>(a.rc) + r0 * N, uint32_t(cnt * N * sizeof(TIn)));
    }
    const long long row = grp * G + g;
    const bool active = row < a.rows;
    int ti;
    asm volatile("mov.b32 %0, %1;" : "=r"(ti) : "r"(t));
    float2 v[P];
    af_load<N, TIn>(v, a, row, ti, active);
    af_compress<N, false>(v, a.ha, a.tw, sm, ti);          // v = I[row]
    if (!BACKWARD) {
      if (active) {
#pragma unroll
        for (int m = 0; m < P; ++m) {
          const float q = v[m].x * v[m].x + v[m].y * v[m].y;
          s_acc += q;
          if (q > 0.f) q_acc += q * logf(q);
        }
      }
    } else {
      // G = -(ln p + E) / S * I, with ln p = ln q - ln S.
#pragma unroll
      for (int m = 0; m < P; ++m) {
        const float q = v[m].x * v[m].x + v[m].y * v[m].y;
        const float w = q > 0.f ? (ln_s_minus_e - logf(q)) * inv_s : 0.f;
        v[m] = cscale(v[m], w);
      }
      af_compress<N, true>(v, a.ha, a.tw, sm, ti);         // v = (A^H G)[row]
      if (active) {
        // v[row] again (from L2), four points at a time to bound live registers.
        const TIn* in = static_cast<const TIn*>(a.rc) + row * N + ti;
#pragma unroll
        for (int m0 = 0; m0 < P; m0 += 4) {
          float2 x[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) x[i] = cmul(load_cached(in + T * (m0 + i)), __ldg(a.ph + ti + T * (m0 + i)));
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float2 b = v[m0 + i];
            gsm[ti + T * (m0 + i)] += 2.f * (b.x * x[i].y - b.y * x[i].x);      // 2 Im(conj(b) x)
          }
          asm volatile("" ::: "memory");
        }
      }
    }
  }

  if (!BACKWARD) {
    __shared__ double red[2][32];
    double s = s_acc, q = q_acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_down_sync(0xffffffffu, s, o);
      q += __shfl_down_sync(0xffffffffu, q, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = s;
      red[1][threadIdx.x >> 5] = q;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double ss = 0.0, qq = 0.0;
      for (int w = 0; w < S::kThreads / 32; ++w) {
        ss += red[0][w];
        qq += red[1][w];
      }
      a.sq_part[2 * blockIdx.x] = ss;
      a.sq_part[2 * blockIdx.x + 1] = qq;
    }
  } else {
    // Groups of one CTA cover the same pulses: add their slices.
    __syncthreads();
    const float* g0 = reinterpret_cast<const float*>(smem_af + G * S::kSmemPerLine);
    float* dst = a.g_part + (long long)blockIdx.x * N;
    for (int i = threadIdx.x; i < N; i += S::kThreads) {
      float acc = 0.f;
#pragma unroll
      for (int gg = 0; gg < G; ++gg) acc += g0[gg * N + i];
      dst[i] = acc;
    }
  }
}

// S and sum q ln q from the per-CTA partials: one block of kAfRedThreads, each
// thread summing a strided share in FP64, then a shuffle and shared-memory
// reduction.
constexpr int kAfRedThreads = 256;

__global__ void __launch_bounds__(kAfRedThreads) af_stats_kernel(const double* __restrict__ sq_part, int grid,
                                                                 double* __restrict__ stats) {
  __shared__ double red[2][kAfRedThreads / 32];
  double s = 0.0, q = 0.0;
  for (int b = threadIdx.x; b < grid; b += kAfRedThreads) {
    s += sq_part[2 * b];
    q += sq_part[2 * b + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    q += __shfl_down_sync(0xffffffffu, q, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s;
    red[1][threadIdx.x >> 5] = q;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s = 0.0;
    q = 0.0;
    for (int w = 0; w < kAfRedThreads / 32; ++w) {
      s += red[0][w];
      q += red[1][w];
    }
    stats[0] = s;
    stats[1] = q;
    stats[2] = s > 0.0 ? log(s) - q / s : 0.0;
    stats[3] = s > 0.0 ? log(s) : 0.0;
  }
}

// grad[i] = sum over CTAs b of g_part[b][i], in FP64: a block covers 32
// consecutive pulses (one per lane: coalesced rows) with 8 warps splitting
// the CTAs between them, then adds the 8 partial sums.
constexpr int kAfGradSlices = 8;

__global__ void __launch_bounds__(32 * kAfGradSlices) af_grad_kernel(const float* __restrict__ g_part, int grid,
                                                                    int n, float* __restrict__ grad) {
  __shared__ double red[kAfGradSlices][32];
  const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  double acc = 0.0;
  if (i < n)
    for (int b = slice; b < grid; b += kAfGradSlices) acc += g_part[(long long)b * n + i];
  red[slice][lane] = acc;
  __syncthreads();
  if (slice == 0 && i < n) {
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < kAfGradSlices; ++k) t += red[k][lane];
    grad[i] = float(t);
  }
}

template <int N, class TIn, bool BACKWARD>
cudaError_t launch_af_n(const AfArgs& a, int* grid_out, cudaStream_t s) {
  using S = RowShape<N>;
  auto kern = af_kernel<N, TIn, BACKWARD>;
  constexpr size_t kBytes = af_smem_bytes<N, BACKWARD>();
  // One-time, thread-safe set-up (function-local static): resident CTAs,
  // capped by the workspace's partial-gradient slots.
  static const LaunchSetup setup = setup_kernel(kern, S::kThreads, kBytes);
  if (setup.err != cudaSuccess) return setup.err;
  const int cap = setup.resident < kAfMaxCtas ? setup.resident : kAfMaxCtas;
  const long long groups = (a.rows + S::G - 1) / S::G;
  const int grid = int(groups < cap ? groups : cap);
  *grid_out = grid;
  kern<<<grid, S::kThreads, kBytes, s>>>(a);
  return cudaGetLastError();
}

template <class TIn, bool BACKWARD>
cudaError_t launch_af(int log2n, const AfArgs& a, int* grid, cudaStream_t s) {
  switch (log2n) {
    case 8: return launch_af_n<256, TIn, BACKWARD>(a, grid, s);
    case 9: return launch_af_n<512, TIn, BACKWARD>(a, grid, s);
    case 10: return launch_af_n<1024, TIn, BACKWARD>(a, grid, s);
    case 11: return launch_af_n<2048, TIn, BACKWARD>(a, grid, s);
    case 12: return launch_af_n<4096, TIn, BACKWARD>(a, grid, s);
    case 13: return launch_af_n<8192, TIn, BACKWARD>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

size_t af_workspace_bytes(long long n_az) {
  return size_t(kAfMaxCtas) * 2 * sizeof(double) + size_t(kAfMaxCtas) * size_t(n_az) * sizeof(float) +
         size_t(n_az) * sizeof(float2) + size_t(kAfMaxCtas) * sizeof(float) + 256;
}

AfWorkspaceLayout af_workspace_layout(void* workspace, long long n_az) {
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  AfWorkspaceLayout l;
  l.sq_part = reinterpret_cast<double*>(ws);
  ws += size_t(kAfMaxCtas) * 2 * sizeof(double);
  l.g_part = reinterpret_cast<float*>(ws);
  ws += size_t(kAfMaxCtas) * size_t(n_az) * sizeof(float);
  l.ph = reinterpret_cast<float2*>(ws);
  ws += size_t(n_az) * sizeof(float2);
  l.q_part = reinterpret_cast<float*>(ws);
  ws += size_t(kAfMaxCtas) * sizeof(float);
  l.qmax = reinterpret_cast<float*>(ws);
  return l;
}

cudaError_t af_phase_table(const float* phi, float2* ph, long long n_az, cudaStream_t s) {
  af_phase_kernel<<<int((n_az + 255) / 256), 256, 0, s>>>(phi, ph, int(n_az));
  return cudaGetLastError();
}

cudaError_t af_entropy_stats(const double* sq_part, int grid, double* stats, cudaStream_t s) {
  af_stats_kernel<<<1, kAfRedThreads, 0, s>>>(sq_part, grid, stats);
  return cudaGetLastError();
}

cudaError_t af_gradient_sum(const float* g_part, int grid, int n_az, float* grad, cudaStream_t s) {
  af_grad_kernel<<<(n_az + 31) / 32, 32 * kAfGradSlices, 0, s>>>(g_part, grid, n_az, grad);
  return cudaGetLastError();
}

cudaError_t launch_autofocus(int log2n, bool rc16, const void* rc, const float* phi, const float2* ha,
                             const float2* tw, long long n_rg, double* stats, float* grad, void* workspace,
                             bool prefetch, cudaStream_t s) {
  const long long n_az = 1LL << log2n;
  const AfWorkspaceLayout l = af_workspace_layout(workspace, n_az);
  AfArgs a;
  a.sq_part = l.sq_part;
  a.g_part = l.g_part;
  float2* ph = l.ph;
  a.rc = rc;
  a.ph = ph;
  a.ha = ha;
  a.tw = tw;
  a.rows = n_rg;
  a.stats = stats;
  a.prefetch = prefetch;
  cudaError_t e = af_phase_table(phi, ph, n_az, s);
  if (e != cudaSuccess) return e;
  int grid = 0;
  e = rc16 ? launch_af<__half2, false>(log2n, a, &grid, s) : launch_af<float2, false>(log2n, a, &grid, s);
  if (e != cudaSuccess) return e;
  if ((e = af_entropy_stats(a.sq_part, grid, stats, s)) != cudaSuccess) return e;
  if (grad == nullptr) return cudaSuccess;
  e = rc16 ? launch_af<__half2, true>(log2n, a, &grid, s) : launch_af<float2, true>(log2n, a, &grid, s);
  if (e != cudaSuccess) return e;
  return af_gradient_sum(a.g_part, grid, int(n_az), grad, s);
}

}  // namespace bfp
