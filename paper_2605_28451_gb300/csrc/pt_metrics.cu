// Point-target quality metrics of a SAR image, in FP64 on the GPU
// (Section VI, Table III: PSLR, ISLR, target SNR, 3 dB resolution).
//
// The paper names the metrics without defining windows; the definitions here
// are the ones the oracle states:
//   - peak cell: argmax |I| within +-4 cells of the nominal target cell;
//   - a 64 x 64 window around it is interpolated x16 by zero-padding its 2-D
//     DFT (frequencies k < 32 kept at k, the others at k - 64);
//   - the interpolated maximum is searched within +-1 cell of the peak cell,
//     and the range and azimuth cuts through it (1024 fine samples each) are
//     evaluated from the window spectrum, separably;
//   - per cut: mainlobe from the peak to the first local minimum on each side,
//     PSLR = 20 log10(max sidelobe / peak), ISLR = 10 log10(sidelobe energy /
//     mainlobe energy), 3 dB width between the half-power crossings (linear
//     interpolation), in original cells;
//   - SNR = 10 log10(|peak|^2 / mean |I|^2) over the cells at least `guard`
//     cells from every target in both axes.
// The FP64 sums run in stages over many CTAs (GB300's FP64 rate is a small
// fraction of its FP32 rate, so one CTA per target leaves most SMs idle):
// window rows, window columns, the fine grid around the peak, the two cuts,
// then the serial cut metrics; targets go through in chunks of kPtChunk with
// their intermediates in the caller's workspace.  Every sum keeps the order
// of the definition's loops.  A separate kernel reduces the noise power in
// FP64.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "pt_metrics.h"

namespace bfp {

namespace {

constexpr int kW = 64;            // window
constexpr int kF = 16;            // interpolation factor
constexpr int kFine = kW * kF;    // 1024 fine samples per axis
constexpr int kThreads = 256;           // noise reduction
constexpr int kSpan = 2 * kF + 1;       // fine samples within +-1 cell of the peak cell, per axis
constexpr int kLo = (kW / 2 - 1) * kF;  // first of them, in fine indices of the window frame
constexpr int kCutParts = 16;           // CTAs per target for the two cuts (2 x 1024 samples)
constexpr int kPtChunk = 16;            // targets per pass of the staged kernels

// One target's intermediates (caller's workspace).
struct PtScratch {
  double2 tmp[kW * kW];     // window rows transformed: [a][kr]
  double2 spec[kW * kW];    // window spectrum S[ka][kr]
  double cut[2 * kFine];    // range cut, then azimuth cut (magnitudes)
  double fine_v[kSpan];     // per fine row ul: the largest |U|^2 ...
  int fine_i[kSpan];        // ... and its column vl
  int peak[2];              // peak cell (eta, r)
  int fine_peak[2];         // interpolated maximum (ua, ur), fine indices of the window frame
};

template <class T> __device__ __forceinline__ double2 pixel(const T* img, long long i);
template <> __device__ __forceinline__ double2 pixel<float2>(const float2* img, long long i) {
  const float2 v = img[i];
  return make_double2(v.x, v.y);
}
template <> __device__ __forceinline__ double2 pixel<__half2>(const __half2* img, long long i) {
  const float2 v = __half22float2(img[i]);
  return make_double2(v.x, v.y);
}

__device__ __forceinline__ double2 cmuld(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 caddd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double mag2(double2 a) { return a.x * a.x + a.y * a.y; }

// exp(sign 2 pi i m / n) in FP64.
__device__ __forceinline__ double2 expi(int sign, long long m, int n) {
  double s, c;
  sincospi(2.0 * double(sign) * double(m % n) / double(n), &s, &c);
  return make_double2(c, s);
}

// Every phase the kernel needs is a multiple of 2 pi / 64 (the window DFT,
// sign -1) or 2 pi / 1024 (the x16 interpolation, sign +1): two tables in
// shared memory, filled once per CTA with expi, replace the per-term
// sincospi of the sums (the sums themselves are unchanged).  n is a power of
// two, so m mod n is m & (n - 1) for negative m too.
struct PhaseTables {
  const double2* fwd64;     // exp(-2 pi i m / 64)
  const double2* inv1024;   // exp(+2 pi i m / 1024)
  __device__ __forceinline__ double2 w64(long long m) const { return fwd64[m & (kW - 1)]; }
  __device__ __forceinline__ double2 w1024(long long m) const { return inv1024[m & (kFine - 1)]; }
};

__device__ __forceinline__ int freq(int k) { return k < kW / 2 ? k : k - kW; }


// The two phase tables, once per call: exp(-2 pi i m / 64), exp(+2 pi i m / 1024).
__global__ void phase_table_kernel(double2* __restrict__ tab) {
  for (int i = threadIdx.x; i < kW + kFine; i += blockDim.x) tab[i] = i < kW ? expi(-1, i, kW) : expi(+1, i - kW, kFine);
}

// Copies the tables into shared memory (kW + kFine entries).
__device__ __forceinline__ PhaseTables load_tables(const double2* __restrict__ g, double2* sh) {
  for (int i = threadIdx.x; i < kW + kFine; i += blockDim.x) sh[i] = g[i];
  __syncthreads();
  return PhaseTables{sh, sh + kW};
}

// Largest (v, -i) over the block: value first, then the smallest index.
__device__ __forceinline__ void argmax_smem(double* v, int* idx, int n) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int b = 0;
    for (int i = 1; i < n; ++i)
      if (v[i] > v[b] || (v[i] == v[b] && idx[i] < idx[b])) b = i;
    v[0] = v[b];
    idx[0] = idx[b];
  }
  __syncthreads();
}

// Stage 1, CTA (a, q), thread kr: the peak cell (argmax |I| within +-4
// cells), then row a of the 64 x 64 window around it transformed along range:
// tmp[a][kr] = sum_r w[a][r] e^{-2 pi i r kr / 64}.
template <class T>
__global__ void __launch_bounds__(kW) pt_rows_kernel(const T* __restrict__ img, long long n_az, long long n_rg,
                                                    const int* __restrict__ targets, const double2* __restrict__ tabs,
                                                    PtScratch* __restrict__ scr) {
  __shared__ double2 tab[kW + kFine];
  __shared__ double2 w[kW];
  __shared__ double cand_v[kW];
  __shared__ int cand_i[kW];
  const int t = threadIdx.x, a = blockIdx.x, q = blockIdx.y;
  PtScratch& sc = scr[q];
  const PhaseTables ph = load_tables(tabs, tab);
  const int eta = targets[2 * q], rr = targets[2 * q + 1];
  double best = -1.0;
  int bi = 0;
  for (int i = t; i < 81; i += kW) {
    const long long ga = ((eta + i / 9 - 4) % n_az + n_az) % n_az;
    const long long gr = ((rr + i % 9 - 4) % n_rg + n_rg) % n_rg;
    const double m = mag2(pixel(img, ga * n_rg + gr));
    if (m > best) {
      best = m;
      bi = i;
    }
  }
  cand_v[t] = best;
  cand_i[t] = bi;
  argmax_smem(cand_v, cand_i, kW);
  const int pa = int(((eta + cand_i[0] / 9 - 4) % n_az + n_az) % n_az);
  const int pr = int(((rr + cand_i[0] % 9 - 4) % n_rg + n_rg) % n_rg);
  if (a == 0 && t == 0) {
    sc.peak[0] = pa;
    sc.peak[1] = pr;
  }
  const long long ga = ((pa - kW / 2 + a) % n_az + n_az) % n_az;
  const long long gr = ((pr - kW / 2 + t) % n_rg + n_rg) % n_rg;
  w[t] = pixel(img, ga * n_rg + gr);
  __syncthreads();
  double2 acc = make_double2(0.0, 0.0);
  for (int r = 0; r < kW; ++r) acc = caddd(acc, cmuld(w[r], ph.w64((long long)r * t)));
  sc.tmp[a * kW + t] = acc;
}

// Stage 2, CTA (ka, q), thread kr: spec[ka][kr] = sum_a tmp[a][kr] e^{-2 pi i a ka / 64}.
__global__ void __launch_bounds__(kW) pt_cols_kernel(const double2* __restrict__ tabs, PtScratch* __restrict__ scr) {
  __shared__ double2 tab[kW + kFine];
  const int kr = threadIdx.x, ka = blockIdx.x;
  PtScratch& sc = scr[blockIdx.y];
  const PhaseTables ph = load_tables(tabs, tab);
  double2 acc = make_double2(0.0, 0.0);
  for (int a = 0; a < kW; ++a) acc = caddd(acc, cmuld(sc.tmp[a * kW + kr], ph.w64((long long)a * ka)));
  sc.spec[ka * kW + kr] = acc;
}

// Stage 3, CTA (ul, q): fine row ua = kLo + ul of the interpolation within
// +-1 cell of the peak cell.  Thread kr forms
//   row[kr] = sum_ka S[ka][kr] e^{2 pi i f(ka) ua / 1024},
// then thread vl the sample U[ua][kLo + vl] = sum_kr row[kr] e^{2 pi i f(kr) (kLo + vl) / 1024};
// the row's largest |U|^2 (smallest vl on ties) goes to the workspace.
__global__ void __launch_bounds__(kW) pt_fine_kernel(const double2* __restrict__ tabs, PtScratch* __restrict__ scr) {
  __shared__ double2 tab[kW + kFine];
  __shared__ double2 row[kW];
  __shared__ double cand_v[kW];
  __shared__ int cand_i[kW];
  const int t = threadIdx.x, ul = blockIdx.x;
  PtScratch& sc = scr[blockIdx.y];
  const PhaseTables ph = load_tables(tabs, tab);
  double2 acc = make_double2(0.0, 0.0);
  for (int ka = 0; ka < kW; ++ka)
    acc = caddd(acc, cmuld(sc.spec[ka * kW + t], ph.w1024((long long)freq(ka) * (kLo + ul))));
  row[t] = acc;
  __syncthreads();
  double m = -1.0;
  if (t < kSpan) {
    double2 u = make_double2(0.0, 0.0);
    for (int kr = 0; kr < kW; ++kr) u = caddd(u, cmuld(row[kr], ph.w1024((long long)freq(kr) * (kLo + t))));
    m = mag2(u);
  }
  cand_v[t] = m;
  cand_i[t] = t;
  argmax_smem(cand_v, cand_i, kW);
  if (t == 0) {
    sc.fine_v[ul] = cand_v[0];
    sc.fine_i[ul] = cand_i[0];
  }
}

// Stage 4, CTA (part, q): the interpolated maximum (ua, ur) over the fine
// rows (largest value, then smallest row), the spectrum's row through ua and
// column through ur, and this CTA's share of the two 1024-sample cuts.
__global__ void __launch_bounds__(2 * kW) pt_cut_kernel(const double2* __restrict__ tabs,
                                                       PtScratch* __restrict__ scr) {
  __shared__ double2 tab[kW + kFine];
  __shared__ double2 vec[2 * kW];             // row[kr], then col[ka]
  __shared__ int fine[2];
  const int t = threadIdx.x;
  PtScratch& sc = scr[blockIdx.y];
  const PhaseTables ph = load_tables(tabs, tab);
  if (t == 0) {
    int b = 0;
    for (int i = 1; i < kSpan; ++i)
      if (sc.fine_v[i] > sc.fine_v[b]) b = i;        // rows in order: ties keep the smaller row
    fine[0] = kLo + b;
    fine[1] = kLo + sc.fine_i[b];
  }
  __syncthreads();
  const int ua = fine[0], ur = fine[1];
  double2 acc = make_double2(0.0, 0.0);
  if (t < kW) {
    for (int ka = 0; ka < kW; ++ka) acc = caddd(acc, cmuld(sc.spec[ka * kW + t], ph.w1024((long long)freq(ka) * ua)));
  } else {
    const int ka = t - kW;
    for (int kr = 0; kr < kW; ++kr) acc = caddd(acc, cmuld(sc.spec[ka * kW + kr], ph.w1024((long long)freq(kr) * ur)));
  }
  vec[t] = acc;
  __syncthreads();
  const double norm = 1.0 / double(kW * kW);
  constexpr int kPer = 2 * kFine / kCutParts;
  for (int i = blockIdx.x * kPer + t; i < (blockIdx.x + 1) * kPer; i += blockDim.x) {
    const int which = i / kFine, u = i % kFine;
    const double2* v = vec + which * kW;
    double2 c = make_double2(0.0, 0.0);
    for (int k = 0; k < kW; ++k) c = caddd(c, cmuld(v[k], ph.w1024((long long)freq(k) * u)));
    sc.cut[i] = sqrt(mag2(c)) * norm;
  }
  if (blockIdx.x == 0 && t == 0) {
    sc.fine_peak[0] = ua;
    sc.fine_peak[1] = ur;
  }
}

// Stage 5, CTA (cut, q), kFinishThreads threads: one cut's metrics with the
// cut in shared memory -- the first maximum and the energy sums reduced over
// the block (largest value, then smallest index; FP64 tree sums), the short
// walks on one thread.  Per cut: mainlobe from the peak to the first local
// minimum on each side, PSLR = 20 log10(max sidelobe / peak), ISLR =
// 10 log10(sidelobe / mainlobe energy), 3 dB width between the half-power
// crossings (linear interpolation), in original cells.
constexpr int kFinishThreads = 256;
__global__ void __launch_bounds__(kFinishThreads) pt_finish_kernel(const PtScratch* __restrict__ scr, int q0,
                                                                  double* __restrict__ out) {
  __shared__ double mag[kFine];
  __shared__ double rv[kFinishThreads], re[kFinishThreads], rm[kFinishThreads];
  __shared__ int ri[kFinishThreads];
  __shared__ int walk[2];
  const int t = threadIdx.x, which = blockIdx.x;
  const PtScratch& sc = scr[blockIdx.y];
  for (int i = t; i < kFine; i += kFinishThreads) mag[i] = sc.cut[which * kFine + i];
  __syncthreads();
  double best = -1.0;
  int bi = 0;
  for (int i = t; i < kFine; i += kFinishThreads)
    if (mag[i] > best) {
      best = mag[i];
      bi = i;
    }
  rv[t] = best;
  ri[t] = bi;
  __syncthreads();
  for (int h = kFinishThreads / 2; h > 0; h >>= 1) {
    if (t < h && (rv[t + h] > rv[t] || (rv[t + h] == rv[t] && ri[t + h] < ri[t]))) {
      rv[t] = rv[t + h];
      ri[t] = ri[t + h];
    }
    __syncthreads();
  }
  const int p = ri[0];
  if (t == 0) {
    int lo = p;
    while (lo > 0 && mag[lo - 1] < mag[lo]) --lo;
    int hi = p;
    while (hi < kFine - 1 && mag[hi + 1] < mag[hi]) ++hi;
    walk[0] = lo;
    walk[1] = hi;
  }
  __syncthreads();
  const int lo = walk[0], hi = walk[1];
  double side_max = 0.0, side_e = 0.0, main_e = 0.0;
  for (int i = t; i < kFine; i += kFinishThreads) {
    const double m2 = mag[i] * mag[i];
    if (i < lo || i > hi) {
      side_max = fmax(side_max, mag[i]);
      side_e += m2;
    } else {
      main_e += m2;
    }
  }
  __syncthreads();                                   // rv / ri are read above until here
  rv[t] = side_max;
  re[t] = side_e;
  rm[t] = main_e;
  __syncthreads();
  for (int h = kFinishThreads / 2; h > 0; h >>= 1) {
    if (t < h) {
      rv[t] = fmax(rv[t], rv[t + h]);
      re[t] += re[t + h];
      rm[t] += rm[t + h];
    }
    __syncthreads();
  }
  if (t != 0) return;
  const bool any_side = lo > 0 || hi < kFine - 1;
  const double pslr = any_side ? 20.0 * log10(rv[0] / mag[p]) : -INFINITY;
  const double islr = any_side ? 10.0 * log10(re[0] / rm[0]) : -INFINITY;
  const double half = 0.5 * mag[p] * mag[p];
  int i = p;
  while (i > lo && mag[i - 1] * mag[i - 1] >= half) --i;
  double left = double(i);
  if (i > 0 && mag[i - 1] * mag[i - 1] < half) {
    const double a = mag[i] * mag[i], b = mag[i - 1] * mag[i - 1];
    left = double(i) - (a - half) / (a - b);
  }
  int j = p;
  while (j < hi && mag[j + 1] * mag[j + 1] >= half) ++j;
  double right = double(j);
  if (j < kFine - 1 && mag[j + 1] * mag[j + 1] < half) {
    const double a = mag[j] * mag[j], b = mag[j + 1] * mag[j + 1];
    right = double(j) + (a - half) / (a - b);
  }
  const double width = (right - left) / double(kF);
  double* o = out + (long long)(q0 + blockIdx.y) * kPtMetricFields;
  if (which == 0) {
    o[kPtPslrRange] = pslr;
    o[kPtIslrRange] = islr;
    o[kPtWidthRange] = width;
    o[kPtPeak] = mag[sc.fine_peak[1]];              // |U| at the interpolated maximum (range cut, sample ur)
    o[kPtPeakAz] = double(sc.peak[0]);
    o[kPtPeakRg] = double(sc.peak[1]);
  } else {
    o[kPtPslrAz] = pslr;
    o[kPtIslrAz] = islr;
    o[kPtWidthAz] = width;
  }
}

// Rows / columns excluded from the noise region: within guard - 1 cells of a
// target (clipped at the image edges, not wrapped).
__global__ void noise_mask_kernel(const int* __restrict__ targets, int k, long long n_az, long long n_rg, int guard,
                                  unsigned char* __restrict__ keep_a, unsigned char* __restrict__ keep_r) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_az) {
    unsigned char keep = 1;
    for (int q = 0; q < k; ++q) {
      const long long d = i - targets[2 * q];
      if (d > -guard && d < guard) keep = 0;
    }
    keep_a[i] = keep;
  }
  if (i < n_rg) {
    unsigned char keep = 1;
    for (int q = 0; q < k; ++q) {
      const long long d = i - targets[2 * q + 1];
      if (d > -guard && d < guard) keep = 0;
    }
    keep_r[i] = keep;
  }
}

// Noise power: mean |I|^2 over the kept rows and columns.  Each CTA takes
// rows a = blockIdx.x, blockIdx.x + gridDim.x, ...; its threads stride the
// row (no division per pixel).  |I|^2 is formed in FP32 (exact products of
// FP16 pixels, one rounding of 2^-24 in the sum), accumulated in FP64; the
// cell count is an integer.
template <class T>
__global__ void __launch_bounds__(kThreads) noise_kernel(const T* __restrict__ img, long long n_az, long long n_rg,
                                                         const unsigned char* __restrict__ keep_a,
                                                         const unsigned char* __restrict__ keep_r,
                                                         double* __restrict__ partial) {
  __shared__ double rs[kThreads], rc[kThreads];
  double s = 0.0;
  long long c = 0;
  for (long long a = blockIdx.x; a < n_az; a += gridDim.x) {
    if (!keep_a[a]) continue;
    const T* row = img + a * n_rg;
    for (long long r = threadIdx.x; r < n_rg; r += kThreads) {
      if (keep_r[r]) {
        const double2 v = pixel(row, r);
        const float x = float(v.x), y = float(v.y);
        s += double(fmaf(x, x, y * y));
        ++c;
      }
    }
  }
  rs[threadIdx.x] = s;
  rc[threadIdx.x] = double(c);
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      rs[threadIdx.x] += rs[threadIdx.x + h];
      rc[threadIdx.x] += rc[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = rs[0];
    partial[2 * blockIdx.x + 1] = rc[0];
  }
}

// The partials reduced by one block (FP64 tree), then each target's SNR.
__global__ void __launch_bounds__(kThreads) snr_kernel(const double* __restrict__ partial, int blocks, int k,
                                                       double* __restrict__ out) {
  __shared__ double rs[kThreads], rc[kThreads];
  double s = 0.0, c = 0.0;
  for (int b = threadIdx.x; b < blocks; b += kThreads) {
    s += partial[2 * b];
    c += partial[2 * b + 1];
  }
  rs[threadIdx.x] = s;
  rc[threadIdx.x] = c;
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      rs[threadIdx.x] += rs[threadIdx.x + h];
      rc[threadIdx.x] += rc[threadIdx.x + h];
    }
    __syncthreads();
  }
  const double noise = rc[0] > 0.0 ? rs[0] / rc[0] : NAN;
  for (int q = threadIdx.x; q < k; q += kThreads) {
    double* o = out + q * kPtMetricFields;
    o[kPtNoise] = noise;
    o[kPtSnr] = 10.0 * log10(o[kPtPeak] * o[kPtPeak] / noise);
  }
}

// Workspace: the noise masks and partial sums, the phase tables, and the
// staged kernels' intermediates for kPtChunk targets.
struct PtLayout {
  size_t keep_a, keep_r, partial, tabs, scratch, total;
};
PtLayout pt_layout(long long n_az, long long n_rg) {
  PtLayout l{};
  l.keep_a = 0;
  l.keep_r = size_t((n_az + 255) / 256) * 256;
  l.partial = l.keep_r + size_t((n_rg + 255) / 256) * 256;
  l.tabs = l.partial + size_t(kPtNoiseBlocks) * 2 * sizeof(double);
  l.scratch = (l.tabs + size_t(kW + kFine) * sizeof(double2) + 255) / 256 * 256;
  l.total = l.scratch + size_t(kPtChunk) * sizeof(PtScratch);
  return l;
}

template <class T>
cudaError_t launch_typed(const void* img, long long n_az, long long n_rg, const int* targets, int k, int guard,
                         double* out, void* ws, cudaStream_t s) {
  const PtLayout l = pt_layout(n_az, n_rg);
  unsigned char* base = static_cast<unsigned char*>(ws);
  unsigned char* keep_a = base + l.keep_a;
  unsigned char* keep_r = base + l.keep_r;
  double* partial = reinterpret_cast<double*>(base + l.partial);
  double2* tabs = reinterpret_cast<double2*>(base + l.tabs);
  PtScratch* scr = reinterpret_cast<PtScratch*>(base + l.scratch);
  cudaError_t e;
  if (k > 0) {
    phase_table_kernel<<<1, 256, 0, s>>>(tabs);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  for (int q0 = 0; q0 < k; q0 += kPtChunk) {
    const int kc = k - q0 < kPtChunk ? k - q0 : kPtChunk;
    pt_rows_kernel<T><<<dim3(kW, kc), kW, 0, s>>>(static_cast<const T*>(img), n_az, n_rg, targets + 2 * q0, tabs, scr);
    pt_cols_kernel<<<dim3(kW, kc), kW, 0, s>>>(tabs, scr);
    pt_fine_kernel<<<dim3(kSpan, kc), kW, 0, s>>>(tabs, scr);
    pt_cut_kernel<<<dim3(kCutParts, kc), 2 * kW, 0, s>>>(tabs, scr);
    pt_finish_kernel<<<dim3(2, kc), kFinishThreads, 0, s>>>(scr, q0, out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const long long longest = n_az > n_rg ? n_az : n_rg;
  noise_mask_kernel<<<int((longest + 255) / 256), 256, 0, s>>>(targets, k, n_az, n_rg, guard, keep_a, keep_r);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  noise_kernel<T><<<kPtNoiseBlocks, kThreads, 0, s>>>(static_cast<const T*>(img), n_az, n_rg, keep_a, keep_r, partial);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  snr_kernel<<<1, kThreads, 0, s>>>(partial, kPtNoiseBlocks, k, out);
  return cudaGetLastError();
}

}  // namespace

size_t pt_workspace_bytes(long long n_az, long long n_rg) { return pt_layout(n_az, n_rg).total; }

cudaError_t launch_point_target_metrics(const void* img, bool img16, long long n_az, long long n_rg,
                                        const int* targets, int k, int guard, double* out, void* ws, cudaStream_t s) {
  return img16 ? launch_typed<__half2>(img, n_az, n_rg, targets, k, guard, out, ws, s)
               : launch_typed<float2>(img, n_az, n_rg, targets, k, guard, out, ws, s);
}

}  // namespace bfp
