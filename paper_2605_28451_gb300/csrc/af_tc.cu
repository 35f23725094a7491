// Entropy autofocus on the tensor-core rows: 4096 pulses per range bin, FP16
// operands at every radix-16 pass, FP32 accumulation (Table IV's "FP16
// multiply, FP32 accumulate" mode applied to the autofocus chain).
//
// The model and the adjoint are those of autofocus.cu:
//   v = rc . e^{-j phi},  I = A v = IDFT(DFT(v) . Ha),  q = |I|^2,
//   G = -(ln(q / S) + E) / S . I,  A^H G = IDFT(DFT(G) . conj(Ha)),
//   dE/dphi[n] = 2 sum_r Im(conj((A^H G)[r][n]) v[r][n]).
// Per range bin the entropy kernel runs six passes (forward, filter into the
// inverse's A tile, inverse) and accumulates S and sum q ln q from the
// accumulators; the gradient kernel runs the same six, writes G as the next
// forward's input, runs six more with conj(Ha), and accumulates the pulse
// gradients in registers: thread tau owns pulses tau + 128 h + 256 q for every
// range bin it processes.
//
// Scaling.  G holds I times (ln S - E - ln q) / S, far below FP16's normal
// range for a large image (1/S).  The kernel stores G' = sigma (ln S - E -
// ln q) I instead, sigma a power of two chosen from the largest q of the
// entropy pass so that |G'| <= 64 (the transform's first two passes grow it
// by at most 256, inside FP16's range), and divides the pulse sums by
// S sigma at the end.  Over q in (0, qmax], |(c - ln q) sqrt(q)| is at most
// sqrt(qmax) (|c| + |ln qmax|) + 2/e, which the bound below covers.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "af_tc.h"
#include "autofocus.h"
#include "tc_fft.cuh"

namespace bfp {

namespace {

constexpr int kAfTcBackwardCtasPerSm = 5;   // 32 gradient registers per thread on top of the passes

struct AfTcArgs {
  RowArgs ra;              // status, pass-major twiddles, DFT-16 matrix
  const void* rc;          // [rows][4096]
  const float2* ph;        // e^{-j phi[n]}
  const float2* ha;        // azimuth filter spectrum
  long long rows;
  const double* stats;     // S, sum q ln q, E, ln S (gradient kernel)
  const float* qmax;       // largest q of the entropy pass (gradient kernel)
  double* sq_part;         // [grid][2] (entropy kernel)
  float* q_part;           // [grid] largest q per CTA (entropy kernel)
  float* g_part;           // [grid][4096] (gradient kernel)
  int prefetch;            // rc in device memory: each CTA prefetches its next row into L2
};

template <class TIn>
__device__ __forceinline__ float2 load_point(const TIn* p);
template <>
__device__ __forceinline__ float2 load_point<__half2>(const __half2* p) {
  return __half22float2(*p);
}
template <>
__device__ __forceinline__ float2 load_point<float2>(const float2* p) {
  return *p;
}

// The last pass of a transform, with the accumulators handed to `epi(h, rho,
// d)` for both M tiles (rows rho = tau and 128 + tau).
template <class Epi>
__device__ __forceinline__ bool tc_last_pass(int* status, uint64_t* bar, uint32_t tmem, uint32_t lane_tmem,
                                             uint32_t a_base, uint32_t b, uint32_t& phase, Epi epi) {
  if (!tc_issue_wait(status, bar, tmem, a_base, b, phase)) return false;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t d[32];
    tc::ld32(lane_tmem + uint32_t(32 * h), d);
    epi(h, int(threadIdx.x) + 128 * h, d);
  }
  tc::fence_before();
  return true;
}

template <class TIn, bool BACKWARD>
__global__ void __launch_bounds__(tc::kThreads, BACKWARD ? kAfTcBackwardCtasPerSm : tc::kCtasPerSm)
af_tc_kernel(const AfTcArgs a) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  unsigned char* sA = smem_tc;
  const float2* s_tw = reinterpret_cast<const float2*>(smem_tc + kTwOff);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_tc + kBarOff);
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t tmem = tc_cta_setup(a.ra.tc_b, a.ra.tw, smem_tc);
  const uint32_t lane_tmem = tmem + (uint32_t(32 * warp) << 16);
  const uint32_t a_base = smem_addr(sA), b_base = smem_addr(smem_tc + kBOff), b_last = b_base + kBBytes;
  const TIn* rc = static_cast<const TIn*>(a.rc);
  uint32_t phase = 0;
  bool ok = true;

  float c0 = 0.f, sigma = 1.f;
  if (BACKWARD) {
    c0 = float(a.stats[3] - a.stats[2]);              // ln S - E
    const float qm = fmaxf(*a.qmax, 1e-30f);
    const float bound = sqrtf(qm) * (fabsf(c0) + fabsf(logf(qm))) + 1.f;
    sigma = exp2f(floorf(log2f(64.f / bound)));
  }
  float s_acc = 0.f, q_acc = 0.f, q_max = 0.f;
  float g_acc[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) g_acc[i] = 0.f;

  for (long long row = blockIdx.x; ok && row < a.rows; row += gridDim.x) {
    const TIn* line = rc + row * kN;
    if (a.prefetch && tid == 0 && row + gridDim.x < a.rows)
      prefetch_l2_bulk(rc + (row + gridDim.x) * kN, uint32_t(kN * sizeof(TIn)));
    // v = rc . e^{-j phi} as the pass-0 input: butterfly j takes pulses j + 256 r.
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = tid + 128 * h;
      uint32_t x[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int n = j + 256 * r;
        const __half2 v = __float22half2_rn(cmul(load_point(line + n), __ldg(a.ph + n)));
        x[r] = *reinterpret_cast<const uint32_t*>(&v);
      }
      tc_store_row0(sA, j, x);
    }
    // I = IDFT(DFT(v) . Ha): forward, filter into A, inverse.
    auto to_filter = [&](int, int rho, const uint32_t(&d)[32]) { tc_filter_to_a<false>(sA, rho, d, a.ha + rho); };
    ok = tc_pass<0, kForward>(a.ra, row, sA, bar, tmem, lane_tmem, a_base, b_base, phase, s_tw) &&
         tc_pass<1, kForward>(a.ra, row, sA, bar, tmem, lane_tmem, a_base, b_base, phase, s_tw) &&
         tc_last_pass(a.ra.status, bar, tmem, lane_tmem, a_base, b_base, phase, to_filter) &&
         tc_pass<0, kForward>(a.ra, row, sA, bar, tmem, lane_tmem, a_base, b_base, phase, s_tw) &&
         tc_pass<1, kForward>(a.ra, row, sA, bar, tmem, lane_tmem, a_base, b_base, phase, s_tw);
    if (!ok) break;
    if constexpr (!BACKWARD) {
      ok = tc_last_pass(a.ra.status, bar, tmem, lane_tmem, a_base, b_last, phase,
                        [&](int, int, const uint32_t(&d)[32]) {
#pragma unroll
                          for (int q = 0; q < 16; ++q) {
                            const float re = __uint_as_float(d[2 * q]), im = __uint_as_float(d[2 * q + 1]);
                            const float qq = re * re + im * im;
                            s_acc += qq;
                            if (qq > 0.f) q_acc += qq * logf(qq);
                            q_max = fmaxf(q_max, qq);
                          }
                        });
    } else {
      // G' = sigma (ln S - E - ln q) I, as the next forward's pass-0 input.
      ok = tc_last_pass(a.ra.status, bar, tmem, lane_tmem, a_base, b_last, phase,
                        [&](int, int rho, const uint32_t(&d)[32]) {
                          uint32_t x[16];
#pragma unroll
                          for (int q = 0; q < 16; ++q) {
                            const float re = __uint_as_float(d[2 * q]), im = __uint_as_float(d[2 * q + 1]);
                            const float qq = re * re + im * im;
                            const float w = qq > 0.f ? sigma * (c0 - logf(qq)) : 0.f;
                            const __half2 g = __floats2half2_rn(w * re, w * im);
                            x[q] = *reinterpret_cast<const uint32_t*>(&g);
                          }
                          tc_store_row0(sA, rho, x);
                        });
      // A^H G' = IDFT(DFT(G') . conj(Ha)); the pulse gradients from it and v.
      auto to_filter_conj = [&](int, int rho, const uint32_t(&d)[32]) {
        tc_filter_to_a<true>(sA, rho, d, a.ha + rho);
      };
      ok = ok && tc_pass<0, kForward>(a.ra, row, sA, bar, tmem, lane_tmem, a_base, b_base, phase, s_tw) &&
           tc_pass<1, kForward>(a.ra, row, sA, bar, tmem, lane_tmem, a_base, b_base, phase, s_tw) &&
           tc_last_pass(a.ra.status, bar, tmem, lane_tmem, a_base, b_base, phase, to_filter_conj) &&
           tc_pass<0, kForward>(a.ra, row, sA, bar, tmem, lane_tmem, a_base, b_base, phase, s_tw) &&
           tc_pass<1, kForward>(a.ra, row, sA, bar, tmem, lane_tmem, a_base, b_base, phase, s_tw) &&
           tc_last_pass(a.ra.status, bar, tmem, lane_tmem, a_base, b_last, phase,
                        [&](int h, int rho, const uint32_t(&d)[32]) {
#pragma unroll
                          for (int q = 0; q < 16; ++q) {
                            const int n = rho + 256 * q;
                            const float2 v = cmul(load_point(line + n), __ldg(a.ph + n));
                            const float bx = __uint_as_float(d[2 * q]), by = __uint_as_float(d[2 * q + 1]);
                            g_acc[16 * h + q] += 2.f * (bx * v.y - by * v.x);     // 2 Im(conj(b) v)
                          }
                        });
    }
  }

  if constexpr (!BACKWARD) {
    __shared__ double red[2][4];
    __shared__ float red_max[4];
    double s = s_acc, q = q_acc;
    float m = q_max;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_down_sync(0xffffffffu, s, o);
      q += __shfl_down_sync(0xffffffffu, q, o);
      m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    }
    if ((tid & 31) == 0) {
      red[0][warp] = s;
      red[1][warp] = q;
      red_max[warp] = m;
    }
    __syncthreads();
    if (tid == 0) {
      a.sq_part[2 * blockIdx.x] = red[0][0] + red[0][1] + red[0][2] + red[0][3];
      a.sq_part[2 * blockIdx.x + 1] = red[1][0] + red[1][1] + red[1][2] + red[1][3];
      a.q_part[blockIdx.x] = fmaxf(fmaxf(red_max[0], red_max[1]), fmaxf(red_max[2], red_max[3]));
    }
  } else {
    // dE/dphi = (1 / (S sigma)) sum 2 Im(conj(A^H G') v): this CTA's share.
    const float scale = float(1.0 / (a.stats[0] * double(sigma)));
    float* dst = a.g_part + (long long)blockIdx.x * kN;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < 16; ++q) dst[tid + 128 * h + 256 * q] = g_acc[16 * h + q] * scale;
  }
  tc_cta_teardown(ok, smem_tc, tmem, phase);
}

// Largest of the per-CTA maxima (one block of 256 threads).
__global__ void af_max_kernel(const float* __restrict__ part, int grid, float* __restrict__ out) {
  __shared__ float red[8];
  float m = 0.f;
  for (int i = threadIdx.x; i < grid; i += blockDim.x) m = fmaxf(m, part[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float r = red[0];
    for (int w = 1; w < 8; ++w) r = fmaxf(r, red[w]);
    *out = r;
  }
}

template <class TIn, bool BACKWARD>
cudaError_t launch_af_tc_kernel(const AfTcArgs& a, int cap, int* grid_out, cudaStream_t s) {
  auto kern = af_tc_kernel<TIn, BACKWARD>;
  // Resident CTAs per SM: the register limit of __launch_bounds__ (TMEM holds
  // at least that many 64-column allocations).  Computed once, thread-safely.
  static const LaunchSetup setup = []() -> LaunchSetup {
    LaunchSetup r{cudaSuccess, 0};
    int dev = 0, sms = 0;
    if ((r.err = cudaGetDevice(&dev)) != cudaSuccess) return r;
    if ((r.err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return r;
    r.resident = (BACKWARD ? kAfTcBackwardCtasPerSm : tc::kCtasPerSm) * sms;
    return r;
  }();
  if (setup.err != cudaSuccess) return setup.err;
  (void)kern;
  const int resident = setup.resident < cap ? setup.resident : cap;
  const int grid = int(a.rows < resident ? a.rows : resident);
  *grid_out = grid;
  if (grid <= 0) return cudaSuccess;
  kern<<<grid, tc::kThreads, tc::kSmemBytes, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_autofocus_tc(bool rc16, const void* rc, const float2* ph, const float2* ha, const RowArgs& ra,
                                long long n_rg, double* stats, float* grad, const AfTcWorkspace& ws, bool prefetch,
                                cudaStream_t s) {
  AfTcArgs a;
  a.ra = ra;
  a.rc = rc;
  a.ph = ph;
  a.ha = ha;
  a.rows = n_rg;
  a.stats = stats;
  a.qmax = ws.qmax;
  a.sq_part = ws.sq_part;
  a.q_part = ws.q_part;
  a.g_part = ws.g_part;
  a.prefetch = prefetch ? 1 : 0;
  int grid = 0;
  cudaError_t e = rc16 ? launch_af_tc_kernel<__half2, false>(a, ws.max_ctas, &grid, s)
                       : launch_af_tc_kernel<float2, false>(a, ws.max_ctas, &grid, s);
  if (e != cudaSuccess) return e;
  if ((e = af_entropy_stats(ws.sq_part, grid, stats, s)) != cudaSuccess) return e;
  af_max_kernel<<<1, 256, 0, s>>>(ws.q_part, grid, ws.qmax);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (grad == nullptr) return cudaSuccess;
  e = rc16 ? launch_af_tc_kernel<__half2, true>(a, ws.max_ctas, &grid, s)
           : launch_af_tc_kernel<float2, true>(a, ws.max_ctas, &grid, s);
  if (e != cudaSuccess) return e;
  return af_gradient_sum(ws.g_part, grid, 4096, grad, s);
}

}  // namespace bfp
