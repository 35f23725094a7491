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
// One CTA per target; a second kernel reduces the noise power in FP64.
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
constexpr int kTargetThreads = 512;     // one CTA per target: 16 warps for its FP64 sums

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

struct CutResult {
  double pslr, islr, width;
};

// Mainlobe walk and metrics of one magnitude cut (serial, one thread).
__device__ CutResult cut_metrics(const double* mag) {
  int p = 0;
  for (int i = 1; i < kFine; ++i)
    if (mag[i] > mag[p]) p = i;
  int lo = p;
  while (lo > 0 && mag[lo - 1] < mag[lo]) --lo;
  int hi = p;
  while (hi < kFine - 1 && mag[hi + 1] < mag[hi]) ++hi;
  double side_max = 0.0, side_e = 0.0, main_e = 0.0;
  for (int i = 0; i < kFine; ++i) {
    const double m2 = mag[i] * mag[i];
    if (i < lo || i > hi) {
      side_max = fmax(side_max, mag[i]);
      side_e += m2;
    } else {
      main_e += m2;
    }
  }
  CutResult r;
  const bool any_side = lo > 0 || hi < kFine - 1;
  r.pslr = any_side ? 20.0 * log10(side_max / mag[p]) : -INFINITY;
  r.islr = any_side ? 10.0 * log10(side_e / main_e) : -INFINITY;
  const double peak2 = mag[p] * mag[p], half = 0.5 * peak2;
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
  r.width = (right - left) / double(kF);
  return r;
}

template <class T>
__global__ void __launch_bounds__(kTargetThreads) target_kernel(const T* __restrict__ img, long long n_az, long long n_rg,
                                                          const int* __restrict__ targets, double* __restrict__ out) {
  extern __shared__ double2 sh[];
  double2* spec = sh;                                   // [64][64] window spectrum S[ka][kr]
  double2* tmp = sh + kW * kW;                          // [64][64] scratch
  double2* tab64 = tmp + kW * kW;                       // [64] phase table
  double2* tab1024 = tab64 + kW;                        // [1024] phase table
  double* cut = reinterpret_cast<double*>(tab1024 + kFine);  // [2][1024] magnitudes
  __shared__ double red_v[kTargetThreads];
  __shared__ int red_i[kTargetThreads];
  __shared__ int peak_cell[2];
  __shared__ int fine_peak[2];
  const int t = threadIdx.x;
  const int eta = targets[2 * blockIdx.x], rr = targets[2 * blockIdx.x + 1];
  for (int i = t; i < kW; i += kTargetThreads) tab64[i] = expi(-1, i, kW);
  for (int i = t; i < kFine; i += kTargetThreads) tab1024[i] = expi(+1, i, kFine);
  const PhaseTables ph{tab64, tab1024};

  // 1. peak cell within +-4 cells
  {
    double best = -1.0;
    int bi = 0;
    for (int i = t; i < 81; i += kTargetThreads) {
      const long long a = ((eta + i / 9 - 4) % n_az + n_az) % n_az;
      const long long r = ((rr + i % 9 - 4) % n_rg + n_rg) % n_rg;
      const double m = mag2(pixel(img, a * n_rg + r));
      if (m > best) {
        best = m;
        bi = i;
      }
    }
    red_v[t] = best;
    red_i[t] = bi;
    __syncthreads();
    if (t == 0) {
      int b = 0;
      for (int i = 1; i < kTargetThreads; ++i)
        if (red_v[i] > red_v[b] || (red_v[i] == red_v[b] && red_i[i] < red_i[b])) b = i;
      peak_cell[0] = int(((eta + red_i[b] / 9 - 4) % n_az + n_az) % n_az);
      peak_cell[1] = int(((rr + red_i[b] % 9 - 4) % n_rg + n_rg) % n_rg);
    }
    __syncthreads();
  }
  const int pa = peak_cell[0], pr = peak_cell[1];

  // 2. window and its 2-D DFT: tmp[a][kr] = sum_r w[a][r] e^{-2 pi i r kr / 64}; spec[ka][kr] = sum_a ...
  for (int i = t; i < kW * kW; i += kTargetThreads) {
    const int a = i / kW, r = i % kW;
    const long long ga = ((pa - kW / 2 + a) % n_az + n_az) % n_az;
    const long long gr = ((pr - kW / 2 + r) % n_rg + n_rg) % n_rg;
    spec[i] = pixel(img, ga * n_rg + gr);             // window, temporarily
  }
  __syncthreads();
  for (int i = t; i < kW * kW; i += kTargetThreads) {
    const int a = i / kW, kr = i % kW;
    double2 acc = make_double2(0.0, 0.0);
    for (int r = 0; r < kW; ++r) acc = caddd(acc, cmuld(spec[a * kW + r], ph.w64((long long)r * kr)));
    tmp[i] = acc;
  }
  __syncthreads();
  for (int i = t; i < kW * kW; i += kTargetThreads) {
    const int ka = i / kW, kr = i % kW;
    double2 acc = make_double2(0.0, 0.0);
    for (int a = 0; a < kW; ++a) acc = caddd(acc, cmuld(tmp[a * kW + kr], ph.w64((long long)a * ka)));
    spec[i] = acc;
  }
  __syncthreads();

  // 3. interpolated maximum within +-1 cell of the peak cell (fine indices
  //    (kW/2 - 1) * kF .. (kW/2 + 1) * kF of the window frame).
  //    U[ua][ur] = (1 / kW^2) sum_ka sum_kr S[ka][kr] e^{2 pi i (f(ka) ua + f(kr) ur) / kFine}
  constexpr int kLo = (kW / 2 - 1) * kF, kSpan = 2 * kF + 1;
  // tmp[ua_local][kr] = sum_ka S[ka][kr] e^{2 pi i f(ka) ua / kFine}, ua = kLo + ua_local
  for (int i = t; i < kSpan * kW; i += kTargetThreads) {
    const int ul = i / kW, kr = i % kW;
    double2 acc = make_double2(0.0, 0.0);
    for (int ka = 0; ka < kW; ++ka)
      acc = caddd(acc, cmuld(spec[ka * kW + kr], ph.w1024((long long)freq(ka) * (kLo + ul))));
    tmp[i] = acc;
  }
  __syncthreads();
  {
    double best = -1.0;
    int bi = 0;
    for (int i = t; i < kSpan * kSpan; i += kTargetThreads) {
      const int ul = i / kSpan, vl = i % kSpan;
      double2 acc = make_double2(0.0, 0.0);
      for (int kr = 0; kr < kW; ++kr)
        acc = caddd(acc, cmuld(tmp[ul * kW + kr], ph.w1024((long long)freq(kr) * (kLo + vl))));
      const double m = mag2(acc);
      if (m > best) {
        best = m;
        bi = i;
      }
    }
    red_v[t] = best;
    red_i[t] = bi;
    __syncthreads();
    if (t == 0) {
      int b = 0;
      for (int i = 1; i < kTargetThreads; ++i)
        if (red_v[i] > red_v[b] || (red_v[i] == red_v[b] && red_i[i] < red_i[b])) b = i;
      fine_peak[0] = kLo + red_i[b] / kSpan;
      fine_peak[1] = kLo + red_i[b] % kSpan;
    }
    __syncthreads();
  }
  const int ua = fine_peak[0], ur = fine_peak[1];
  const double norm = 1.0 / double(kW * kW);

  // 4. the two cuts: range (ua fixed, all ur) and azimuth (ur fixed, all ua)
  //    row[kr] = sum_ka S[ka][kr] e^{2 pi i f(ka) ua / kFine}; col[ka] = sum_kr S[ka][kr] e^{...f(kr) ur}
  double2* row = tmp;
  double2* col = tmp + kW;
  if (t < kW) {
    double2 acc = make_double2(0.0, 0.0);
    for (int ka = 0; ka < kW; ++ka)
      acc = caddd(acc, cmuld(spec[ka * kW + t], ph.w1024((long long)freq(ka) * ua)));
    row[t] = acc;
  } else if (t < 2 * kW) {
    const int ka = t - kW;
    double2 acc = make_double2(0.0, 0.0);
    for (int kr = 0; kr < kW; ++kr)
      acc = caddd(acc, cmuld(spec[ka * kW + kr], ph.w1024((long long)freq(kr) * ur)));
    col[ka] = acc;
  }
  __syncthreads();
  for (int i = t; i < 2 * kFine; i += kTargetThreads) {
    const int which = i / kFine, u = i % kFine;
    const double2* v = which == 0 ? row : col;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < kW; ++k) acc = caddd(acc, cmuld(v[k], ph.w1024((long long)freq(k) * u)));
    cut[i] = sqrt(mag2(acc)) * norm;
  }
  __syncthreads();
  if (t < 2) {
    const CutResult c = cut_metrics(cut + t * kFine);
    double* o = out + blockIdx.x * kPtMetricFields;
    if (t == 0) {
      o[kPtPslrRange] = c.pslr;
      o[kPtIslrRange] = c.islr;
      o[kPtWidthRange] = c.width;
      o[kPtPeak] = cut[ur];                          // |U| at the interpolated maximum
      o[kPtPeakAz] = double(pa);
      o[kPtPeakRg] = double(pr);
    } else {
      o[kPtPslrAz] = c.pslr;
      o[kPtIslrAz] = c.islr;
      o[kPtWidthAz] = c.width;
    }
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

template <class T>
__global__ void __launch_bounds__(kThreads) noise_kernel(const T* __restrict__ img, long long n_az, long long n_rg,
                                                         const unsigned char* __restrict__ keep_a,
                                                         const unsigned char* __restrict__ keep_r,
                                                         double* __restrict__ partial) {
  __shared__ double rs[kThreads], rc[kThreads];
  double s = 0.0, c = 0.0;
  const long long total = n_az * n_rg;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < total; i += (long long)gridDim.x * kThreads) {
    const long long a = i / n_rg, r = i - a * n_rg;
    if (keep_a[a] && keep_r[r]) {
      s += mag2(pixel(img, i));
      c += 1.0;
    }
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
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = rs[0];
    partial[2 * blockIdx.x + 1] = rc[0];
  }
}

__global__ void snr_kernel(const double* __restrict__ partial, int blocks, int k, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double s = 0.0, c = 0.0;
  for (int b = 0; b < blocks; ++b) {
    s += partial[2 * b];
    c += partial[2 * b + 1];
  }
  const double noise = c > 0.0 ? s / c : NAN;
  for (int q = 0; q < k; ++q) {
    double* o = out + q * kPtMetricFields;
    o[kPtNoise] = noise;
    o[kPtSnr] = 10.0 * log10(o[kPtPeak] * o[kPtPeak] / noise);
  }
}

template <class T>
cudaError_t launch_typed(const void* img, long long n_az, long long n_rg, const int* targets, int k, int guard,
                         double* out, void* ws, cudaStream_t s) {
  const size_t smem = size_t(2 * kW * kW + kW + kFine) * sizeof(double2) + size_t(2 * kFine) * sizeof(double);
  auto kern = target_kernel<T>;
  // Set once per instantiation, thread-safely (function-local static).
  static const cudaError_t setup = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (setup != cudaSuccess) return setup;
  kern<<<k, kTargetThreads, smem, s>>>(static_cast<const T*>(img), n_az, n_rg, targets, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  unsigned char* keep_a = static_cast<unsigned char*>(ws);
  unsigned char* keep_r = keep_a + ((n_az + 255) / 256) * 256;
  double* partial = reinterpret_cast<double*>(keep_r + ((n_rg + 255) / 256) * 256);
  const long long longest = n_az > n_rg ? n_az : n_rg;
  noise_mask_kernel<<<int((longest + 255) / 256), 256, 0, s>>>(targets, k, n_az, n_rg, guard, keep_a, keep_r);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  noise_kernel<T><<<kPtNoiseBlocks, kThreads, 0, s>>>(static_cast<const T*>(img), n_az, n_rg, keep_a, keep_r, partial);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  snr_kernel<<<1, 32, 0, s>>>(partial, kPtNoiseBlocks, k, out);
  return cudaGetLastError();
}

}  // namespace

size_t pt_workspace_bytes(long long n_az, long long n_rg) {
  return size_t((n_az + 255) / 256) * 256 + size_t((n_rg + 255) / 256) * 256 + size_t(kPtNoiseBlocks) * 2 * sizeof(double);
}

cudaError_t launch_point_target_metrics(const void* img, bool img16, long long n_az, long long n_rg,
                                        const int* targets, int k, int guard, double* out, void* ws, cudaStream_t s) {
  return img16 ? launch_typed<__half2>(img, n_az, n_rg, targets, k, guard, out, ws, s)
               : launch_typed<float2>(img, n_az, n_rg, targets, k, guard, out, ws, s);
}

}  // namespace bfp
