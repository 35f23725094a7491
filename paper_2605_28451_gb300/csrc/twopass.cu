// Long lines (N = N1 x 256, N1 = 128 or 256: 32768 and 65536 points) as two
// streaming passes with no waits between CTAs -- the four-step factorisation
// of Section V's batched transforms, with n = n2 + 256 n1 and k = k1 + N1 k2:
//
//   X[k1 + N1 k2] = sum_n2 W_256^{n2 k2} W_N^{n2 k1} sum_n1 x[n2 + 256 n1] W_N1^{n1 k1}
//
// Pass A (columns).  A CTA takes C = 256 / T1 consecutive columns n2 of one
// line (T1 = N1 / 16 threads per column; 16 columns at N1 = 256, 32 at 128):
// for every n1 its threads read the C columns' points as one contiguous
// segment (64 or 128 bytes in FP16), run the N1-point DFT of each column in
// registers and shared memory, multiply by W_N^{n2 k1} (a [k1][n2] table,
// consecutive lanes on consecutive n2) and write the intermediate
// Y[k1][n2] at the same positions, again as contiguous segments.
// Pass B (rows).  A CTA takes 16 consecutive rows k1 of the intermediate: each
// row's 256 points are contiguous; after the 256-point DFT the results are
// staged in shared memory as [k2][row] and written so that a half-warp's 16
// values X[k1 + N1 k2], k1 = 16 r .. 16 r + 15, form one contiguous segment.
//
// The inverse takes conj(x) / N on load and conjugates on store (Eq. 1).
// Arithmetic is FP32; the intermediate is stored as FP16 for FP16 storage
// (one more FP16 rounding, at the pass boundary) and as FP32 otherwise.
// Lines are dense (line l at l N) or at the point offsets of an uneven plan.  With the batch cut into chunks of a few hundred lines the
// intermediate of a chunk stays in L2 between the two passes.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "fft_rows.cuh"
#include "twopass.h"

namespace bfp {

namespace {

// The intermediate: FP16 for FP16 storage (one more FP16 rounding, at the
// pass boundary, as an FP16 exchange makes), FP32 otherwise -- FP8 outputs
// must stay the rounding of an FP32 result.
template <class TS> struct ScratchOf { using T = float2; };
template <> struct ScratchOf<__half2> { using T = __half2; };

__device__ __forceinline__ long long line_base(const TwoPassArgs& a, long long line, int n) {
  return a.line_off != nullptr ? a.line_off[line] : line * (long long)n;
}

template <int N1, class TS, int MODE, bool SCALED>
__global__ void __launch_bounds__(256, 4) twopass_columns_kernel(const TwoPassArgs a) {
  constexpr int N = N1 * 256, P = kPointsPerThread, T1 = N1 / P, C = 256 / T1;
  using TScr = typename ScratchOf<TS>::T;
  extern __shared__ float2 smem_tp[];
  const int col = threadIdx.x % C;
  const int t = threadIdx.x / C;
  const int tiles = 256 / C;
  const long long line = a.first_line + blockIdx.x / tiles;
  const int n2 = (blockIdx.x % tiles) * C + col;
  const long long base = line_base(a, line, N);
  if (a.pf_ahead > 0 && threadIdx.x == 0) {
    // The CTA pf_ahead blocks later reads one column tile of its line; the
    // tiles of a line together cover it, so each CTA prefetches its share of
    // that line as one contiguous range (N / tiles points).
    const long long blk = blockIdx.x + a.pf_ahead;
    if (blk / tiles < a.count) {
      const long long b2 = line_base(a, a.first_line + blk / tiles, N) + (blk % tiles) * (long long)(N / tiles);
      prefetch_l2_bulk(static_cast<const TS*>(a.in) + b2, uint32_t(size_t(N / tiles) * sizeof(TS)));
    }
  }
  const TS* in = static_cast<const TS*>(a.in) + base + n2;
  float2 v[P];
#pragma unroll
  for (int m = 0; m < P; ++m) {
    float2 x = Storage<TS>::load(in + 256 * (t + T1 * m));
    if (SCALED) x = cscale(x, a.in_scale);
    if (MODE == kInverse) x = cscale(cconj(x), 1.0f / float(N));
    v[m] = x;
  }
  line_dft<N1>(v, a.tw_col, smem_tp + col * pad16(N1), t);
  TScr* y = static_cast<TScr*>(a.scratch) + (line - a.first_line) * (long long)N + n2;
#pragma unroll
  for (int m = 0; m < P; ++m) {
    const int k1 = t + T1 * m;
    const float2 w = __ldg(a.tw_4step + k1 * 256 + n2);
    Storage<TScr>::store(y + 256 * k1, k1 == 0 ? v[m] : cmul(v[m], w));
  }
}

template <int N1, class TS, int MODE, bool SCALED>
__global__ void __launch_bounds__(256, 4) twopass_rows_kernel(const TwoPassArgs a) {
  constexpr int N = N1 * 256, P = kPointsPerThread, T = 256 / P, R = 16;   // 16 rows of 16 threads
  using TScr = typename ScratchOf<TS>::T;
  extern __shared__ float2 smem_tp[];
  const int row = threadIdx.x / T;
  const int t = threadIdx.x % T;
  const int tiles = N1 / R;
  const long long line = a.first_line + blockIdx.x / tiles;
  const int k1_0 = (blockIdx.x % tiles) * R;
  const TScr* y =
      static_cast<const TScr*>(a.scratch) + (line - a.first_line) * (long long)N + (k1_0 + row) * 256;
  if (a.pf_ahead > 0 && threadIdx.x == 0) {
    // The CTA pf_ahead blocks later reads 16 contiguous rows of the intermediate.
    const long long blk = blockIdx.x + a.pf_ahead;
    if (blk / tiles < a.count) {
      const TScr* p2 = static_cast<const TScr*>(a.scratch) + (blk / tiles) * (long long)N + (blk % tiles) * R * 256;
      prefetch_l2_bulk(p2, uint32_t(size_t(R) * 256 * sizeof(TScr)));
    }
  }
  float2 v[P];
#pragma unroll
  for (int m = 0; m < P; ++m) v[m] = Storage<TScr>::load(y + t + T * m);
  line_dft<256>(v, a.tw_row, smem_tp + row * pad16(256), t);
  // Stage [k2][row] (17 slots per k2: conflict-free) and store 16 rows of one
  // k2 as one contiguous segment of the output.
  float2* st = smem_tp;
  __syncthreads();   // the last pass read the exchange buffers
#pragma unroll
  for (int m = 0; m < P; ++m) st[(t + T * m) * (R + 1) + row] = v[m];
  __syncthreads();
  const long long base = line_base(a, line, N);
  TS* out = static_cast<TS*>(a.out) + base + k1_0;
  const int r = threadIdx.x % R;
  const int k2_0 = threadIdx.x / R;      // 0 .. 15
#pragma unroll
  for (int m = 0; m < P; ++m) {
    const int k2 = k2_0 + 16 * m;
    float2 x = st[k2 * (R + 1) + r];
    if (MODE == kInverse) x = cconj(x);
    if (SCALED) x = cscale(x, a.out_scale);
    v[m] = x;
    Storage<TS>::store(out + r + (long long)N1 * k2, x);
  }
  check_finite<Storage<TS>, P>(a.finite_flag, [&](int m) { return v[m]; });
}

template <int N1, class TS, int MODE, bool SCALED>
cudaError_t launch_twopass_typed(const TwoPassArgs& a, cudaStream_t s) {
  constexpr int T1 = N1 / kPointsPerThread, C = 256 / T1;
  constexpr size_t kColBytes = size_t(C) * pad16(N1) * sizeof(float2);
  constexpr size_t kRowBytes = size_t(16) * pad16(256) * sizeof(float2);
  static_assert(size_t(256) * 17 * sizeof(float2) <= kRowBytes, "staging fits the row buffers");
  auto ka = twopass_columns_kernel<N1, TS, MODE, SCALED>;
  auto kb = twopass_rows_kernel<N1, TS, MODE, SCALED>;
  static const LaunchSetup sa = setup_kernel(ka, 256, kColBytes);
  static const LaunchSetup sb = setup_kernel(kb, 256, kRowBytes);
  if (sa.err != cudaSuccess) return sa.err;
  if (sb.err != cudaSuccess) return sb.err;
  if (a.lines <= 0) return cudaSuccess;
  const long long chunk = a.chunk_lines > 0 ? a.chunk_lines : a.lines;
  for (long long l0 = 0; l0 < a.lines; l0 += chunk) {
    TwoPassArgs b = a;
    b.first_line = a.first_line + l0;
    const long long cnt = a.lines - l0 < chunk ? a.lines - l0 : chunk;
    b.count = cnt;
    b.pf_ahead = a.pf_ahead > 0 ? sa.resident : 0;
    ka<<<dim3(unsigned(cnt * (256 / C))), 256, kColBytes, s>>>(b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    b.pf_ahead = a.pf_ahead > 0 ? sb.resident : 0;
    kb<<<dim3(unsigned(cnt * (N1 / 16))), 256, kRowBytes, s>>>(b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int N1, class TS>
cudaError_t launch_twopass_mode(int mode, bool scaled, const TwoPassArgs& a, cudaStream_t s) {
  if (mode == kForward) {
    return scaled ? launch_twopass_typed<N1, TS, kForward, true>(a, s)
                  : launch_twopass_typed<N1, TS, kForward, false>(a, s);
  }
  return scaled ? launch_twopass_typed<N1, TS, kInverse, true>(a, s)
                : launch_twopass_typed<N1, TS, kInverse, false>(a, s);
}

template <class TS>
cudaError_t launch_twopass_len(int log2n, int mode, bool scaled, const TwoPassArgs& a, cudaStream_t s) {
  switch (log2n) {
    case 15: return launch_twopass_mode<128, TS>(mode, scaled, a, s);
    case 16: return launch_twopass_mode<256, TS>(mode, scaled, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

size_t twopass_scratch_bytes(int kind, long long lines_per_chunk, int log2n) {
  return size_t(lines_per_chunk) * (size_t(1) << log2n) * (kind == 1 ? sizeof(__half2) : sizeof(float2));
}

cudaError_t launch_twopass(int kind, int log2n, int mode, const TwoPassArgs& a, cudaStream_t s) {
  switch (kind) {
    case 0: return launch_twopass_len<float2>(log2n, mode, false, a, s);
    case 1: return launch_twopass_len<__half2>(log2n, mode, false, a, s);
    case 2: return launch_twopass_len<Fp8x2<E4M3>>(log2n, mode, true, a, s);
    case 3: return launch_twopass_len<Fp8x2<E5M2>>(log2n, mode, true, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bfp
