// Range-Doppler imaging with range-cell migration correction and a
// range-dependent azimuth filter (Section VI's RCMC stage of the range-Doppler
// chain, on the paper's FP16 block-floating-point transforms).
//
// For a target at slant range R seen with the hyperbolic range history
// sqrt(R^2 + v^2 t^2), at Doppler frequency f it sits dR(f) = R (1/D(f) - 1)
// further out, D(f) = sqrt(1 - (lambda f / (2 v))^2), and its azimuth chirp
// has the FM rate k_a(R) = 2 v^2 / (lambda R PRF^2) cycles per pulse^2.  The
// line kernels here are the two steps the migration-free chain lacks:
//
//   rcmc_rows       one line per Doppler bin f, along range: the band-limited
//                   shift of the line by s = dR(f, R0) / range_cell cells back
//                   towards near range, as DFT, a linear phase
//                   exp(+2 pi i q s / N) on the signed frequency q (the Nyquist
//                   bin takes cos(pi s)), 1/N shift and inverse (Eq. 1's
//                   schedule; s is computed per line in FP64 from the geometry);
//   azimuth_rows    one line per range bin r, along Doppler: the bin's own
//                   matched filter H_r = conj(DFT(ref_r)) (optionally divided by
//                   max |DFT(ref_r)|), ref_r the chirp exp(-i pi k_a(R_r) n^2),
//                   n in [-L/2, L/2), circularly centred at index 0, generated
//                   and transformed in registers (its phase reduced modulo 2 pi
//                   in FP64), then H_r times the line, the 1/N shift and the
//                   inverse.  No table of n_rg filters is read from HBM.
//
// Both run the radix-16 Stockham line transform of fft_rows.cuh in FP32
// registers; storage is FP16 (half2) or FP32 (float2).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "fft_rows.cuh"
#include "rda.h"

namespace bfp {

namespace {

constexpr double kPiD = 3.14159265358979323846;

template <int N, class TIn, class TOut, bool AZIMUTH>
__global__ void __launch_bounds__(RowShape<N>::kThreads, RowShape<N>::kThreads >= 512 ? 1 : 2)
rda_rows_kernel(const RdaArgs a) {
  using S = RowShape<N>;
  constexpr int P = S::P, T = S::T, G = S::G;
  extern __shared__ float2 smem_rda[];
  __shared__ float warp_max[32];
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const long long line = (long long)blockIdx.x * G + g;
  const bool active = line < a.lines;
  float2* sm = smem_rda + g * S::kSmemPerLine;
  const float inv_n = 1.0f / float(N);
  float2 h[P];
  if constexpr (AZIMUTH) {
    // The line's reference chirp, phase pi k_a n^2 reduced modulo 2 pi in FP64.
    const double r_m = a.range_dependent ? a.geo.centre_range_m + (double(line) - 0.5 * double(a.other)) *
                                                                      a.geo.range_cell_m
                                         : a.geo.centre_range_m;
    const double ka = 2.0 * a.geo.speed_mps * a.geo.speed_mps /
                      (a.geo.wavelength_m * r_m * a.geo.prf_hz * a.geo.prf_hz);
    const int half = a.aperture / 2;
#pragma unroll
    for (int m = 0; m < P; ++m) {
      const int i = t + T * m;
      const int n = i < N / 2 ? i : i - N;
      if (n >= -half && n < a.aperture - half) {
        double x = ka * double(n) * double(n);   // phase / pi
        x -= 2.0 * floor(0.5 * x);               // in [0, 2)
        float s, c;
        sincospif(-float(x), &s, &c);
        h[m] = make_float2(c, s);
      } else {
        h[m] = make_float2(0.f, 0.f);
      }
    }
    line_dft<N>(h, a.tw, sm, t);
    __syncthreads();   // the exchange buffer is reused by the data transform
    float scale = 1.0f;
    if (a.peak_normalise) {
      float mx = 0.f;
#pragma unroll
      for (int m = 0; m < P; ++m) mx = fmaxf(mx, h[m].x * h[m].x + h[m].y * h[m].y);
      if constexpr (T < 32) {
#pragma unroll
        for (int o = T / 2; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      } else {
        constexpr int W = T / 32;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = mx;
        __syncthreads();
        mx = 0.f;
#pragma unroll
        for (int w = 0; w < W; ++w) mx = fmaxf(mx, warp_max[g * W + w]);
      }
      scale = mx > 0.f ? rsqrtf(mx) : 1.0f;
    }
#pragma unroll
    for (int m = 0; m < P; ++m) h[m] = make_float2(h[m].x * scale, -h[m].y * scale);   // conj
  } else {
    // Bulk RCMC of Doppler bin `line` (signed index k): move the line back by
    // dR(f, R0) / range_cell cells, y(r) = x(r + s), as exp(+2 pi i q s / N).
    const long long k = line < a.other / 2 ? line : line - a.other;
    const double f = double(k) * a.geo.prf_hz / double(a.other);
    const double u = a.geo.wavelength_m * f / (2.0 * a.geo.speed_mps);
    const double s = a.geo.centre_range_m * (1.0 / sqrt(1.0 - u * u) - 1.0) / a.geo.range_cell_m;
    const float sf = float(s);
#pragma unroll
    for (int m = 0; m < P; ++m) {
      const int q = t + T * m;
      if (q == N / 2) {
        h[m] = make_float2(cospif(sf), 0.f);
      } else {
        const int qs = q < N / 2 ? q : q - N;
        float sn, cs;
        sincospif(2.0f * float(qs) * sf * inv_n, &sn, &cs);
        h[m] = make_float2(cs, sn);
      }
    }
  }
  float2 v[P];
  if (active) {
    const TIn* in = static_cast<const TIn*>(a.in) + line * (long long)N + t;
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = Storage<TIn>::load(in + T * m);
  } else {
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = make_float2(0.f, 0.f);
  }
  if constexpr (!AZIMUTH) line_dft<N>(v, a.tw, sm, t);   // the azimuth lines arrive as spectra
  // filter, then the inverse as conj(DFT(conj(.) / N)) (Eq. 1)
#pragma unroll
  for (int m = 0; m < P; ++m) v[m] = cscale(cconj(cmul(v[m], h[m])), inv_n);
  int t2;
  asm volatile("mov.b32 %0, %1;" : "=r"(t2) : "r"(t));
  line_dft<N>(v, a.tw, sm, t2);
  if (active) {
    TOut* out = static_cast<TOut*>(a.out) + line * (long long)N + t;
#pragma unroll
    for (int m = 0; m < P; ++m) Storage<TOut>::store(out + T * m, cconj(v[m]));
  }
}

template <int N, class TS, bool AZIMUTH>
cudaError_t launch_rda_n(const RdaArgs& a, cudaStream_t s) {
  using S = RowShape<N>;
  auto kern = rda_rows_kernel<N, TS, TS, AZIMUTH>;
  static const LaunchSetup setup = setup_kernel(kern, S::kThreads, S::kSmemBytes);
  if (setup.err != cudaSuccess) return setup.err;
  if (a.lines <= 0) return cudaSuccess;
  const long long grid = (a.lines + S::G - 1) / S::G;
  kern<<<dim3(unsigned(grid)), dim3(S::kThreads), S::kSmemBytes, s>>>(a);
  return cudaGetLastError();
}

template <class TS, bool AZIMUTH>
cudaError_t launch_rda_typed(int log2n, const RdaArgs& a, cudaStream_t s) {
  switch (log2n) {
    case 8: return launch_rda_n<256, TS, AZIMUTH>(a, s);
    case 9: return launch_rda_n<512, TS, AZIMUTH>(a, s);
    case 10: return launch_rda_n<1024, TS, AZIMUTH>(a, s);
    case 11: return launch_rda_n<2048, TS, AZIMUTH>(a, s);
    case 12: return launch_rda_n<4096, TS, AZIMUTH>(a, s);
    case 13: return launch_rda_n<8192, TS, AZIMUTH>(a, s);
    case 14: return launch_rda_n<16384, TS, AZIMUTH>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_rcmc_rows(int log2n, bool f16, const RdaArgs& a, cudaStream_t s) {
  return f16 ? launch_rda_typed<__half2, false>(log2n, a, s) : launch_rda_typed<float2, false>(log2n, a, s);
}

cudaError_t launch_azimuth_rows(int log2n, bool f16, const RdaArgs& a, cudaStream_t s) {
  return f16 ? launch_rda_typed<__half2, true>(log2n, a, s) : launch_rda_typed<float2, true>(log2n, a, s);
}

}  // namespace bfp
