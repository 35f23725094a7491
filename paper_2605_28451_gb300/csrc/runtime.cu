// Plans, twiddle tables, argument checking and the C ABI of include/bfpfft.h.
//
// Nothing here does arithmetic of the method except the twiddle generator
// (FP64 sincospi on the GPU, rounded once to FP32) and the small filter
// normalisation kernel; every transform runs in the row kernels of
// fft_rows.cuh, launched through launch.h.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <string>
#include <cstdio>
#include <sys/stat.h>
#include <vector>
#include <algorithm>

#include "bfpfft.h"
#include "launch.h"
#include "metrics.h"
#include "af_tc.h"
#include "autofocus.h"
#include "uneven.h"
#include "pt_metrics.h"
#include "rda.h"
#include "twopass.h"

namespace {

constexpr int kMinLog2 = 4;
constexpr int kMaxLog2 = 16;       // plain transforms; SAR and autofocus lines stop earlier
constexpr int kSarMaxLog2 = 14;

int log2_exact(int64_t n) {
  if (n <= 0 || (n & (n - 1)) != 0) return -1;
  int l = 0;
  while ((int64_t(1) << l) < n) ++l;
  return l;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// True for device memory.  Inputs elsewhere (pinned host buffers that the
// kernels read in place over the CPU-GPU link) get no bulk L2 prefetch.
bool device_memory(const void* p) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice;
}

// The variant to use when the input is not device memory: no bulk L2
// prefetch of it, and no bulk (TMA) copies from it -- the same exchange with
// plain loads instead.
int without_l2(int variant) {
  switch (variant) {
    case bfp::kRowsPlainL2: return bfp::kRowsPlain;
    case bfp::kRowsPlain4L2:
    case bfp::kRowsTma: return bfp::kRowsPlain4;
    case bfp::kRowsTmaPP: return bfp::kRowsPlainPP;
    case bfp::kRowsPlainHL2:
    case bfp::kRowsPlainH4L2:
    case bfp::kRowsPlainHS4L2:
    case bfp::kRowsTmaH: return bfp::kRowsPlainH;
    case bfp::kRowsTmaHPP: return bfp::kRowsPlainHPP;
    default: return variant;
  }
}

// Variants whose exchanges round to FP16 (FP16 storage only); with one of
// them, lines of 8192 points or more by the four-step kernel also exchange
// their rows as FP16 words.
bool fp16_exchange_variant(int variant) {
  switch (variant) {
    case bfp::kRowsPlainH:
    case bfp::kRowsPlainHPP:
    case bfp::kRowsTmaH:
    case bfp::kRowsTmaHPP:
    case bfp::kRowsPlainHL2:
    case bfp::kRowsPlainH4L2:
    case bfp::kRowsPlainHS4L2: return true;
    default: return false;
  }
}

// Host-side fault injection for the error paths: BFPFFT_FAULT=plan|alloc|launch
// makes the named step fail without touching the GPU.
bool fault(const char* step) {
  const char* f = std::getenv("BFPFFT_FAULT");
  return f != nullptr && std::strcmp(f, step) == 0;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return BFPFFT_OK;
  if (e == cudaErrorMemoryAllocation) return BFPFFT_ERR_OOM;
  return BFPFFT_ERR_CUDA;
}

// Pass-major twiddle table of a length-n transform (radix-16 passes, the last
// one radix n / Ns): for every pass after the first, with sub-length Ns and
// radix R, entry (Ns - 16) + (r - 1) Ns + k holds W_{Ns R}^{k r} =
// exp(-2 pi i k r / (Ns R)) for r in [1, R), k in [0, Ns).  Evaluated in FP64
// (sincospi of an exact dyadic fraction) and rounded once to FP32.
__global__ void twiddle_kernel(float2* tw, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 16) return;
  int ns = 16;
  while (ns * 16 < n && i >= ns * 16 - 16) ns *= 16;
  const int radix = (n / ns) >= 16 ? 16 : n / ns;
  const int local = i - (ns - 16);
  const int r = local / ns + 1;
  const int k = local - (r - 1) * ns;
  double s, c;
  sincospi(-2.0 * double(k * r) / double(ns * radix), &s, &c);
  tw[i] = make_float2(float(c), float(s));
}

// Four-step twiddles of a length n = N1 * 4096 line: T[k1][n2] = W_n^{n2 k1}
// for k1 < N1, n2 < 4096 (n entries, k1-major so that lanes with consecutive
// n2 read consecutive entries).  FP64 sincospi, rounded once to FP32.
__global__ void fourstep_twiddle_kernel(float2* tw, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k1 = i / 4096, n2 = i % 4096;
  double s, c;
  sincospi(-2.0 * double((long long)n2 * k1) / double(n), &s, &c);
  tw[i] = make_float2(float(c), float(s));
}

// Two-pass twiddles of a length n = N1 * 256 line: T[k1][n2] = W_n^{n2 k1} for
// k1 < N1, n2 < 256 (n entries; consecutive lanes take consecutive n2).  FP64
// sincospi, rounded once to FP32.
__global__ void twopass_twiddle_kernel(float2* tw, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k1 = i / 256, n2 = i % 256;
  double s, c;
  sincospi(-2.0 * double((long long)n2 * k1) / double(n), &s, &c);
  tw[i] = make_float2(float(c), float(s));
}

// Per-device, per-length twiddle tables, created on first use and kept for
// the life of the process (a few hundred KB per device at most).  Keys
// 0..16: pass-major Stockham tables; 100 + log2 n: four-step tables;
// 500 + log2 n: two-pass tables.
std::mutex g_tw_mutex;
std::map<std::pair<int, int>, float2*> g_tw;

int get_twiddles(int log2n, float2** out) {
  *out = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  std::lock_guard<std::mutex> lock(g_tw_mutex);
  auto it = g_tw.find({dev, log2n});
  if (it != g_tw.end()) {
    *out = it->second;
    return BFPFFT_OK;
  }
  if (fault("alloc")) return BFPFFT_ERR_OOM;
  const bool two = log2n >= 500;
  const bool four = !two && log2n >= 100;
  const int n = 1 << (two ? log2n - 500 : four ? log2n - 100 : log2n);
  float2* tw = nullptr;
  e = cudaMalloc(&tw, sizeof(float2) * n);
  if (e != cudaSuccess) return cuda_status(e);
  if (two) {
    twopass_twiddle_kernel<<<(n + 255) / 256, 256>>>(tw, n);
  } else if (four) {
    fourstep_twiddle_kernel<<<(n + 255) / 256, 256>>>(tw, n);
  } else {
    twiddle_kernel<<<(n + 255) / 256, 256>>>(tw, n);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(tw);
    return cuda_status(e);
  }
  g_tw[{dev, log2n}] = tw;
  *out = tw;
  return BFPFFT_OK;
}

// 16-bit twiddle tables (pairs w, wp per entry, 8 bytes) for the rows computed
// in FP16 or bfloat16 arithmetic, cached like the FP32 tables under keys
// 200 + log2 n (FP16) and 300 + log2 n (bfloat16).
int get_twiddles16(int log2n, bool bf16, const void** out) {
  *out = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  const int key = (bf16 ? 300 : 200) + log2n;
  std::lock_guard<std::mutex> lock(g_tw_mutex);
  auto it = g_tw.find({dev, key});
  if (it != g_tw.end()) {
    *out = it->second;
    return BFPFFT_OK;
  }
  if (fault("alloc")) return BFPFFT_ERR_OOM;
  const int n = 1 << log2n;
  float2* tw = nullptr;   // n entries of 8 bytes
  e = cudaMalloc(&tw, sizeof(float2) * n);
  if (e != cudaSuccess) return cuda_status(e);
  e = bfp::launch_twiddles16(tw, n, bf16);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(tw);
    return cuda_status(e);
  }
  g_tw[{dev, key}] = tw;
  *out = tw;
  return BFPFFT_OK;
}

// One device status word per device (bounded device-side waits record
// BFPFFT_ERR_TIMEOUT here); read and cleared by bfpfft_device_status().
std::map<int, int*> g_status;

int get_status_word(int** out) {
  *out = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  std::lock_guard<std::mutex> lock(g_tw_mutex);
  auto it = g_status.find(dev);
  if (it != g_status.end()) {
    *out = it->second;
    return BFPFFT_OK;
  }
  int* w = nullptr;
  e = cudaMalloc(&w, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(w, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_status(e);
  g_status[dev] = w;
  *out = w;
  return BFPFFT_OK;
}

// Corner turns of the SAR calls: "split" (default) compresses dense rows and
// turns the result with a tiled transpose through stream-ordered scratch;
// "fused" turns on chip through cluster distributed shared memory.
// BFPFFT_SAR_TURN selects; the split form measured faster on GB300 (4096 x
// 4096, FP16: 97 us against 120 us per compression).
bool sar_split_turns() {
  const char* v = std::getenv("BFPFFT_SAR_TURN");
  return v == nullptr || std::strcmp(v, "fused") != 0;
}

// Stream-ordered scratch from a library-owned pool per device that keeps its
// memory between calls (release threshold: never), so repeated calls neither
// synchronise nor return memory to the driver.
cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t s) {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  if (fault("alloc")) return cudaErrorMemoryAllocation;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = pools.find(dev);
    if (it == pools.end()) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
      uint64_t keep = UINT64_MAX;
      if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) return e;
      pools[dev] = pool;
    } else {
      pool = it->second;
    }
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

// Row-kernel variant from BFPFFT_ROWS (tma, plain, pp, h16, h16pp, tma_pp,
// tma_h16, tma_h16pp, tc, plain4, plain_l2, plain4_l2).  Unset: plain4_l2,
// the plain kernel with an FP32 exchange at 4 CTAs per SM whose CTAs prefetch
// into L2 the lines of the CTA one resident wave later -- the fastest
// exact-numerics variant measured on GB300; unknown names: the pipelined
// kernel.
int rows_variant() {
  const char* v = std::getenv("BFPFFT_ROWS");
  if (v == nullptr) return bfp::kRowsPlain4L2;
  static const struct { const char* name; int code; } kNames[] = {
      {"tma", bfp::kRowsTma},         {"plain", bfp::kRowsPlain},    {"pp", bfp::kRowsPlainPP},
      {"h16", bfp::kRowsPlainH},      {"h16pp", bfp::kRowsPlainHPP}, {"tma_pp", bfp::kRowsTmaPP},
      {"tma_h16", bfp::kRowsTmaH},    {"tma_h16pp", bfp::kRowsTmaHPP}, {"tc", bfp::kRowsTc},
      {"plain4", bfp::kRowsPlain4},   {"plain_l2", bfp::kRowsPlainL2}, {"plain4_l2", bfp::kRowsPlain4L2},
      {"h16_l2", bfp::kRowsPlainHL2}, {"h16_4_l2", bfp::kRowsPlainH4L2}, {"h16s_4_l2", bfp::kRowsPlainHS4L2},
      {"twopass", bfp::kRowsTwoPass}};
  for (const auto& k : kNames)
    if (std::strcmp(v, k.name) == 0) return k.code;
  return bfp::kRowsTma;
}

// The 16-point DFT matrix of the tensor-core variant in real form, FP16,
// [n][k]: B[2q][2r] = Re W, B[2q][2r+1] = -Im W, B[2q+1][2r] = Im W,
// B[2q+1][2r+1] = Re W with W = exp(-2 pi i q r / 16); one copy per device.
std::map<int, void*> g_tc_b;

int get_tc_matrix(void** out) {
  *out = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  std::lock_guard<std::mutex> lock(g_tw_mutex);
  auto it = g_tc_b.find(dev);
  if (it != g_tc_b.end()) {
    *out = it->second;
    return BFPFFT_OK;
  }
  __half host[32 * 32];
  const double pi = 3.14159265358979323846;
  for (int q = 0; q < 16; ++q)
    for (int r = 0; r < 16; ++r) {
      const double ang = -2.0 * pi * double((q * r) % 16) / 16.0;
      const double wr = std::cos(ang), wi = std::sin(ang);
      host[(2 * q) * 32 + 2 * r] = __double2half(wr);
      host[(2 * q) * 32 + 2 * r + 1] = __double2half(-wi);
      host[(2 * q + 1) * 32 + 2 * r] = __double2half(wi);
      host[(2 * q + 1) * 32 + 2 * r + 1] = __double2half(wr);
    }
  void* d = nullptr;
  e = cudaMalloc(&d, sizeof(host));
  if (e == cudaSuccess) e = cudaMemcpy(d, host, sizeof(host), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (d) cudaFree(d);
    return cuda_status(e);
  }
  g_tc_b[dev] = d;
  *out = d;
  return BFPFFT_OK;
}

// Lines of 8192 points and more use the four-step kernel: the 4096-point
// row table and the four-step table of their length.
int fourstep_tables(int log2n, bfp::RowArgs* a) {
  a->tw_line = nullptr;
  a->tw_4step = nullptr;
  if (log2n < 13) return BFPFFT_OK;
  float2* t = nullptr;
  int st = get_twiddles(12, &t);
  if (st != BFPFFT_OK) return st;
  a->tw_line = t;
  st = get_twiddles(100 + log2n, &t);
  if (st != BFPFFT_OK) return st;
  a->tw_4step = t;
  return BFPFFT_OK;
}

// Common RowArgs set-up: twiddles, status word, unit scales.
int row_args(int log2n, bfp::RowArgs* a) {
  std::memset(a, 0, sizeof(*a));
  int st = get_twiddles(log2n, const_cast<float2**>(&a->tw));
  if (st != BFPFFT_OK) return st;
  st = get_status_word(&a->status);
  if (st != BFPFFT_OK) return st;
  a->in_scale = 1.f;
  a->out_scale = 1.f;
  a->variant = rows_variant();
  return fourstep_tables(log2n, a);
}

bool valid_dtype(int d) { return d >= BFPFFT_F32 && d <= BFPFFT_BF16; }

// H = conj(H) / max_k |H[k]| (or conj only), one CTA.
__global__ void conj_normalise_kernel(float2* h, int n, int peak_normalise) {
  __shared__ float red[1024];
  float m = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float2 v = h[i];
    m = fmaxf(m, v.x * v.x + v.y * v.y);
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  const float scale = (peak_normalise && red[0] > 0.f) ? 1.0f / sqrtf(red[0]) : 1.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float2 v = h[i];
    h[i] = make_float2(v.x * scale, -v.y * scale);
  }
}

}  // namespace

struct bfpfft_plan_s {
  int64_t n;
  int64_t batch;
  int log2n;
  int dtype;
  int direction;
  int device;
  float2* tw;          // shared table from the per-device cache (not owned)
  int* status;         // the plan's own device status word (owned): timeouts, non-finite outputs
  int flags = 0;       // BFPFFT_CHECK_FINITE
  int arith = 0;       // enum bfpfft_arith: the arithmetic the transforms run in
  int in_exp;
  int out_exp;
  int variant = -1;     // row-kernel variant chosen by the tuner (-1: library default)
  // Uneven plans (bfpfft_plan_create_many): owned device arrays.
  bool many = false;
  int tuned_clusters = 0;               // persistent clusters chosen by the tuner (0: all resident)
  int long_twopass = 0;                 // lines of 32768 / 65536 points by the two-pass kernels (1) or in the
                                        // persistent kernel's four-step lines (0)
  int fs_h16 = 0;                       // FP16 storage: four-step lines exchange their rows as FP16 words (1)
  int per_length = 0;                   // one dense-row launch per length over its listed lines (1) instead of
                                        // the persistent kernel
  int has_fourstep = 0;                 // some line has 8192 points or more
  long long len_first[kMaxLog2 + 1] = {};   // lines of 2^l points: first index into d_line_off ...
  long long len_count[kMaxLog2 + 1] = {};   // ... and count
  const float2* tw_len[kMaxLog2 + 1] = {};  // per-length twiddle tables (device pointers, shared cache)
  cudaStream_t side = nullptr;          // one launch per length: the shorter lengths' stream (owned) ...
  cudaEvent_t ev_fork = nullptr;        // ... forked from the caller's stream ...
  cudaEvent_t ev_join = nullptr;        // ... and joined back into it
  int first_short_task = 0;             // first task of a length below 32768
  long long long_first[2] = {0, 0};     // lines of 65536 / 32768 points: first index into d_line_off ...
  long long long_count[2] = {0, 0};     // ... and count
  int kind = 0;                         // storage kind of the persistent kernel
  long long* d_line_off = nullptr;
  bfp::UnevenTask* d_tasks = nullptr;
  const float2** d_tw = nullptr;
  const float2** d_tw4 = nullptr;
  int* d_counter = nullptr;
  int num_tasks = 0;
  int clusters = 0;
  // Graph cache of bfpfft_exec_graph.
  cudaGraphExec_t graph = nullptr;
  const void* graph_in = nullptr;
  void* graph_out = nullptr;
  void* graph_stream_key = nullptr;
};

namespace {

void free_plan_resources(bfpfft_plan p) {
  if (p->graph) cudaGraphExecDestroy(p->graph);
  if (p->status) cudaFree(p->status);
  if (p->d_line_off) cudaFree(p->d_line_off);
  if (p->d_tasks) cudaFree(p->d_tasks);
  if (p->d_tw) cudaFree(p->d_tw);
  if (p->d_tw4) cudaFree(p->d_tw4);
  if (p->d_counter) cudaFree(p->d_counter);
  if (p->side) cudaStreamDestroy(p->side);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
}

// The plan's status word: one device int, zeroed.
int alloc_plan_status(int** out) {
  *out = nullptr;
  int* w = nullptr;
  cudaError_t e = cudaMalloc(&w, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(w, 0, sizeof(int));
  if (e != cudaSuccess) {
    if (w) cudaFree(w);
    return cuda_status(e);
  }
  *out = w;
  return BFPFFT_OK;
}

// Wait self-test: one warp arms an mbarrier for 16 bytes that no copy will
// ever deliver and waits for it with the bounded wait every kernel of the
// library uses; the bound expires, BFPFFT_ERR_TIMEOUT goes to `status` and
// the kernel returns.  Nothing is in flight when it exits.
__global__ void wait_selftest_kernel(int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    bfp::mbar_init(&bar, 1);
    bfp::fence_proxy_async_shared();
    bfp::mbar_arrive_expect_tx(&bar, 16);
  }
  __syncthreads();
  bfp::mbar_wait_bounded(&bar, 0, status);
}

int uneven_kind(int dtype) {
  switch (dtype) {
    case BFPFFT_F32: return 0;
    case BFPFFT_F16_BFP: return 1;
    case BFPFFT_E4M3_BFP: return 2;
    case BFPFFT_E5M2_BFP: return 3;
    default: return -1;
  }
}

}  // namespace

// Lines of 2^log2n points (15 or 16) by the two-pass kernels: `lines` lines,
// dense (line_off nullptr) or at line_off[0 .. lines).  The intermediate goes
// through pool scratch in chunks whose footprint stays near 64 MB, so a chunk's
// intermediate is still in L2 when the second pass reads it.
static int run_twopass(int kind, int log2n, int mode, const void* in, void* out, const long long* line_off,
                       long long lines, float in_scale, float out_scale, int* finite_flag, cudaStream_t s) {
  if (lines <= 0) return BFPFFT_OK;
  bfp::TwoPassArgs t{};
  float2* tab = nullptr;
  int st = get_twiddles(log2n - 8, &tab);
  if (st != BFPFFT_OK) return st;
  t.tw_col = tab;
  if ((st = get_twiddles(8, &tab)) != BFPFFT_OK) return st;
  t.tw_row = tab;
  if ((st = get_twiddles(500 + log2n, &tab)) != BFPFFT_OK) return st;
  t.tw_4step = tab;
  long long chunk = (64ll << 20) / (long long)bfp::twopass_scratch_bytes(kind, 1, log2n);
  if (const char* c = std::getenv("BFPFFT_TWOPASS_CHUNK")) chunk = std::max(1ll, std::atoll(c));
  chunk = std::min(chunk, lines);
  void* scratch = nullptr;
  cudaError_t e = scratch_alloc(&scratch, bfp::twopass_scratch_bytes(kind, chunk, log2n), s);
  if (e != cudaSuccess) return cuda_status(e);
  t.in = in;
  t.out = out;
  t.scratch = scratch;
  t.line_off = line_off;
  t.lines = lines;
  t.chunk_lines = chunk;
  t.in_scale = in_scale;
  t.out_scale = out_scale;
  t.finite_flag = finite_flag;
  t.pf_ahead = device_memory(in) ? 1 : 0;   // L2 prefetch one resident wave ahead (device memory only)
  e = bfp::launch_twopass(kind, log2n, mode, t, s);
  const cudaError_t f = cudaFreeAsync(scratch, s);
  return cuda_status(e != cudaSuccess ? e : f);
}

extern "C" int bfpfft_exec(bfpfft_plan plan, const void* in, void* out, void* stream);

// An uneven plan as one launch per length, longest first: each length's
// lines, listed by their offsets, run the dense-row kernel of a uniform plan
// of that length (the four-step kernel for 32768 / 65536 points, one CTA per
// line for 8192 / 16384, CTA-local groups below), which the persistent
// kernel cannot use because its CTAs are sized for every length at once.
// With FP8 storage each length keeps the block exponents of its uniform plan.
// Lines of 32768 / 65536 points run on the caller's stream, the shorter
// lengths on the plan's side stream forked from it (an event each way, so a
// stream capture takes both branches), so that their launches overlap.
static int exec_per_length(bfpfft_plan plan, const void* in, void* out, cudaStream_t s) {
  const bool dev_mem = device_memory(in);
  const int mode = plan->direction == BFPFFT_INVERSE ? bfp::kInverse : bfp::kForward;
  bool has_long = false, has_short = false;
  for (int l = kMinLog2; l <= kMaxLog2; ++l)
    if (plan->len_count[l] > 0) (l >= 15 ? has_long : has_short) = true;
  const bool fork = has_long && has_short && plan->side != nullptr;
  if (fork) {
    cudaError_t e = cudaEventRecord(plan->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->side, plan->ev_fork, 0);
    if (e != cudaSuccess) return cuda_status(e);
  }
  int result = BFPFFT_OK;
  for (int l = kMaxLog2; l >= kMinLog2 && result == BFPFFT_OK; --l) {
    if (plan->len_count[l] == 0) continue;
    const cudaStream_t ls = fork && l < 15 ? plan->side : s;
    bfp::RowArgs a{};
    a.in = in;
    a.out = out;
    a.tw = plan->tw_len[l];
    a.status = plan->status;
    a.finite_flag = (plan->flags & BFPFFT_CHECK_FINITE) ? plan->status : nullptr;
    a.variant = dev_mem ? bfp::kRowsPlain4L2 : bfp::kRowsPlain4;
    a.no_prefetch = dev_mem ? 0 : 1;
    a.lines = plan->len_count[l];
    a.in_stride = a.out_stride = 1LL << l;
    a.line_off = plan->d_line_off + plan->len_first[l];
    a.fs_h16 = plan->kind == 1 && plan->fs_h16;
    const float sc = float(1 << ((l + 1) / 2));       // FP8 block exponent of a uniform plan of this length
    a.in_scale = plan->kind >= 2 && mode == bfp::kInverse ? sc : 1.f;
    a.out_scale = plan->kind >= 2 && mode == bfp::kForward ? 1.f / sc : 1.f;
    result = fourstep_tables(l, &a);
    if (result != BFPFFT_OK) break;
    cudaError_t e;
    switch (plan->kind) {
      case 0: e = bfp::launch_rows_f32(l, mode, a, ls); break;
      case 1: e = bfp::launch_rows_f16(l, mode, false, a, ls); break;
      default: e = bfp::launch_rows_fp8(l, mode, plan->kind - 2, a, ls); break;
    }
    if (e != cudaSuccess) result = cuda_status(e);
  }
  if (fork) {   // joined whatever happened, so that a capture stays well formed
    cudaError_t e = cudaEventRecord(plan->ev_join, plan->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, plan->ev_join, 0);
    if (e != cudaSuccess && result == BFPFFT_OK) result = cuda_status(e);
  }
  return result;
}

static int exec_many(bfpfft_plan plan, const void* in, void* out, cudaStream_t s) {
  if (plan->per_length) return exec_per_length(plan, in, out, s);
  bfp::UnevenArgs a{};
  a.in = in;
  a.out = out;
  a.line_off = plan->d_line_off;
  a.tasks = plan->d_tasks;
  a.num_tasks = plan->num_tasks;
  const int variant = rows_variant();   // the _l2 row variants also prefetch the next task into L2
  // BFPFFT_ROWS=twopass forces the split (tests); otherwise the tuner's choice.
  const bool forced = std::getenv("BFPFFT_ROWS") != nullptr && variant == bfp::kRowsTwoPass;
  if ((plan->long_twopass || forced) && plan->first_short_task > 0) {
    // Long lines first, by the two-pass kernels; the persistent kernel then
    // takes the tasks of the shorter lengths only.
    const int mode = plan->direction == BFPFFT_INVERSE ? bfp::kInverse : bfp::kForward;
    for (int c = 0; c < 2; ++c) {
      const int l = 16 - c;
      const float sc = float(1 << ((l + 1) / 2));    // FP8 block exponent of a uniform plan of this length
      const bool fp8 = plan->kind >= 2;
      const int st = run_twopass(plan->kind, l, mode, in, out, plan->d_line_off + plan->long_first[c],
                                 plan->long_count[c], fp8 && mode == bfp::kInverse ? sc : 1.f,
                                 fp8 && mode == bfp::kForward ? 1.f / sc : 1.f,
                                 (plan->flags & BFPFFT_CHECK_FINITE) ? plan->status : nullptr, s);
      if (st != BFPFFT_OK) return st;
    }
    a.tasks = plan->d_tasks + plan->first_short_task;
    a.num_tasks = plan->num_tasks - plan->first_short_task;
    if (a.num_tasks == 0) return BFPFFT_OK;
  }
  a.tw = plan->d_tw;
  a.tw4 = plan->d_tw4;
  a.counter = plan->d_counter;
  a.status = plan->status;
  a.finite_flag = (plan->flags & BFPFFT_CHECK_FINITE) ? plan->status : nullptr;
  // BFPFFT_ROWS naming an FP16-exchange variant forces the FP16 row exchange
  // of four-step lines (tests); otherwise the tuner's choice.
  a.fs_h16 = plan->kind == 1 && (plan->fs_h16 || (std::getenv("BFPFFT_ROWS") != nullptr &&
                                                  fp16_exchange_variant(variant)));
  a.prefetch = (variant == bfp::kRowsPlainL2 || variant == bfp::kRowsPlain4L2 || variant == bfp::kRowsPlainHL2 ||
                variant == bfp::kRowsPlainH4L2 || variant == bfp::kRowsPlainHS4L2 || variant == bfp::kRowsTwoPass) &&
               device_memory(in);
  const int want = plan->tuned_clusters > 0 ? plan->tuned_clusters : plan->clusters;
  const int clusters = std::min(want, std::max(1, a.num_tasks));
  return cuda_status(bfp::launch_uneven(plan->kind, plan->direction == BFPFFT_INVERSE, a, clusters, s));
}

// ---------------------------------------------------------------------------
// Autotuner.  Times candidate kernels on the plan's own shape (scratch
// buffers, 2 warm-up and 5 timed launches, median) and keeps the fastest.
// Results are cached in memory and in a text file (BFPFFT_TUNE_CACHE, default
// $HOME/.cache/bfpfft/tune.txt), one "key value ms" line per shape, the key
// naming the GPU, length(s), batch class, dtype and direction.
// BFPFFT_TUNE: off (never tune automatically), cached (apply cached results
// at plan creation), full (also time shapes missing from the cache).
namespace {

std::mutex g_tune_mutex;
std::map<std::string, std::pair<int, float>> g_tune;
bool g_tune_loaded = false;

std::string tune_path() {
  const char* p = std::getenv("BFPFFT_TUNE_CACHE");
  if (p != nullptr && *p) return p;
  const char* home = std::getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/bfpfft/tune.txt";
}

void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  FILE* f = std::fopen(tune_path().c_str(), "r");
  if (f == nullptr) return;
  char key[512];
  int v = 0;
  float ms = 0.f;
  while (std::fscanf(f, "%511s %d %f", key, &v, &ms) == 3) g_tune[key] = {v, ms};
  std::fclose(f);
}

void tune_store_locked() {
  const std::string path = tune_path();
  const size_t slash = path.find_last_of('/');
  if (slash != std::string::npos) {
    std::string dir = path.substr(0, slash);
    // create the directory chain if needed (best effort)
    for (size_t i = 1; i <= dir.size(); ++i)
      if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
  }
  const std::string tmp = path + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (f == nullptr) return;
  for (const auto& kv : g_tune) std::fprintf(f, "%s %d %.5f\n", kv.first.c_str(), kv.second.first, kv.second.second);
  std::fclose(f);
  std::rename(tmp.c_str(), path.c_str());
}

std::string tune_key(bfpfft_plan p) {
  cudaDeviceProp prop;
  std::string gpu = "gpu";
  if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) gpu = prop.name;
  for (auto& c : gpu)
    if (c == ' ') c = '_';
  char buf[256];
  if (p->many) {
    std::snprintf(buf, sizeof(buf), "%s/many/tasks%d/d%d/%s", gpu.c_str(), p->num_tasks, p->dtype,
                  p->direction == BFPFFT_FORWARD ? "fwd" : "inv");
  } else {
    int bclass = 0;
    while ((int64_t(1) << bclass) < p->batch) ++bclass;
    std::snprintf(buf, sizeof(buf), "%s/n%lld/b%d/d%d/%s", gpu.c_str(), (long long)p->n, bclass, p->dtype,
                  p->direction == BFPFFT_FORWARD ? "fwd" : "inv");
  }
  return buf;
}

size_t storage_bytes(int dtype) {
  switch (dtype) {
    case BFPFFT_F32: return 8;
    case BFPFFT_F16_BFP:
    case BFPFFT_F16_NAIVE:
    case BFPFFT_F16_ADAPTIVE:
    case BFPFFT_BF16: return 4;
    default: return 2;
  }
}

}  // namespace

extern "C" int bfpfft_plan_tune(bfpfft_plan plan, int allow_fp16_exchange, int* chosen, float* best_ms) {
  if (plan == nullptr || chosen == nullptr) return BFPFFT_ERR_INVALID_ARG;
  *chosen = -1;
  if (best_ms) *best_ms = 0.f;
  // Adaptive exponents and 16-bit or tensor-core arithmetic run one kernel each: nothing to choose.
  if (plan->batch == 0 || plan->dtype == BFPFFT_F16_ADAPTIVE || plan->arith != BFPFFT_ARITH_F32) return BFPFFT_OK;
  // Scratch: a bounded sample of the plan's own shape.
  int64_t points = 0;
  int64_t sample_batch = plan->batch;
  if (plan->many) {
    // every line of an uneven plan: the last task's line ends the buffer extent
    std::vector<long long> off(1);
    points = 0;
    // extent = max(offset + n) is not stored; use tasks: sum of 65536 points per task is an upper bound
    points = int64_t(plan->num_tasks) * bfp::kUnevenTaskPoints;
    long long max_off = 0;
    std::vector<long long> host_off(size_t(plan->batch));
    if (cudaMemcpy(host_off.data(), plan->d_line_off, sizeof(long long) * host_off.size(),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
      return BFPFFT_ERR_CUDA;
    for (long long o : host_off) max_off = std::max(max_off, o);
    points = std::max<int64_t>(points, max_off + 65536);
  } else {
    sample_batch = std::min<int64_t>(plan->batch, std::max<int64_t>(1, (int64_t(1) << 28) / plan->n));
    points = sample_batch * plan->n;
  }
  const size_t bytes = size_t(points) * storage_bytes(plan->dtype);
  void* in = nullptr;
  void* out = nullptr;
  cudaError_t e = cudaMalloc(&in, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&out, bytes);
  if (e == cudaSuccess) e = cudaMemset(in, 0, bytes);
  if (e != cudaSuccess) {
    if (in) cudaFree(in);
    if (out) cudaFree(out);
    return cuda_status(e);
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int64_t saved_batch = plan->batch;
  const int saved_variant = plan->variant;
  const int saved_clusters = plan->tuned_clusters;
  if (!plan->many) plan->batch = sample_batch;
  std::vector<int> candidates;
  const int saved_long = plan->long_twopass;
  const int saved_fs_h16 = plan->fs_h16;
  const int saved_per_length = plan->per_length;
  if (plan->many) {
    // Uneven plans: the persistent cluster count; whether lines of 32768 /
    // 65536 points run as four-step lines inside the persistent kernel or as
    // the two-pass kernels before it; with allow_fp16_exchange and FP16
    // storage, whether four-step lines exchange their rows as FP16 words
    // (code = clusters + 65536 * two-pass + 131072 * FP16 row exchange).
    const bool has_long = plan->first_short_task > 0;
    const bool h16 = allow_fp16_exchange && plan->kind == 1 && plan->has_fourstep;
    const size_t per_count = size_t(1 + (has_long ? 1 : 0)) * (h16 ? 2 : 1);
    for (int c = plan->clusters; c >= 1 && candidates.size() + per_count <= (h16 ? 12u : 8u); c = c * 3 / 4) {
      for (int mode = 0; mode < 4; ++mode) {
        if (((mode & 1) && !has_long) || ((mode & 2) && !h16)) continue;
        candidates.push_back(c + 65536 * mode);
      }
    }
    // One launch per length (code bit 18; the cluster count does not apply).
    candidates.push_back(plan->clusters + 262144);
    if (h16) candidates.push_back(plan->clusters + 262144 + 131072);
  } else if (plan->log2n >= 15) {
    candidates = {bfp::kRowsPlain4L2, bfp::kRowsTwoPass};
    // four-step lines with the FP16 row exchange
    if (allow_fp16_exchange && plan->dtype == BFPFFT_F16_BFP) candidates.push_back(bfp::kRowsPlainHL2);
  } else {
    candidates = {bfp::kRowsPlain4L2, bfp::kRowsPlainL2, bfp::kRowsPlain, bfp::kRowsPlain4,
                  bfp::kRowsTma,        bfp::kRowsPlainPP, bfp::kRowsTmaPP};
    if (allow_fp16_exchange && (plan->dtype == BFPFFT_F16_BFP || plan->dtype == BFPFFT_F16_NAIVE)) {
      candidates.push_back(bfp::kRowsPlainHS4L2);
      candidates.push_back(bfp::kRowsPlainHL2);
      candidates.push_back(bfp::kRowsPlainH);
      candidates.push_back(bfp::kRowsPlainHPP);
      candidates.push_back(bfp::kRowsTmaH);
      candidates.push_back(bfp::kRowsTmaHPP);
      if (plan->log2n == 12) candidates.push_back(bfp::kRowsTc);
    }
  }
  int st = BFPFFT_OK;
  int best = -1;
  float best_t = 1e30f;
  for (int c : candidates) {
    if (plan->many) {
      plan->tuned_clusters = c & 0xffff;
      plan->long_twopass = (c >> 16) & 1;
      plan->fs_h16 = (c >> 17) & 1;
      plan->per_length = (c >> 18) & 1;
    } else {
      plan->variant = c;
    }
    float ts[5];
    for (int r = 0; r < 7 && st == BFPFFT_OK; ++r) {
      cudaEventRecord(e0, nullptr);
      st = plan->many ? exec_many(plan, in, out, nullptr) : bfpfft_exec(plan, in, out, nullptr);
      cudaEventRecord(e1, nullptr);
      if (cudaEventSynchronize(e1) != cudaSuccess) st = BFPFFT_ERR_CUDA;
      if (r >= 2) cudaEventElapsedTime(&ts[r - 2], e0, e1);
    }
    if (st != BFPFFT_OK) break;
    std::sort(ts, ts + 5);
    if (ts[2] < best_t) {
      best_t = ts[2];
      best = c;
    }
  }
  plan->batch = saved_batch;
  if (plan->many) {
    plan->tuned_clusters = saved_clusters;
    plan->long_twopass = saved_long;
    plan->fs_h16 = saved_fs_h16;
    plan->per_length = saved_per_length;
  } else {
    plan->variant = saved_variant;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(in);
  cudaFree(out);
  if (st != BFPFFT_OK) return st;
  if (plan->many) {
    plan->tuned_clusters = best & 0xffff;
    plan->long_twopass = (best >> 16) & 1;
    plan->fs_h16 = (best >> 17) & 1;
    plan->per_length = (best >> 18) & 1;
  } else {
    plan->variant = best;
  }
  if (plan->graph) {   // a captured graph holds the old schedule
    cudaGraphExecDestroy(plan->graph);
    plan->graph = nullptr;
  }
  *chosen = best;
  if (best_ms) *best_ms = best_t;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  tune_load_locked();
  g_tune[tune_key(plan)] = {best, best_t};
  tune_store_locked();
  return BFPFFT_OK;
}

namespace {

// Plan-creation hook: apply a cached choice, or tune when BFPFFT_TUNE=full.
void tune_on_create(bfpfft_plan p) {
  const char* mode = std::getenv("BFPFFT_TUNE");
  if (mode == nullptr || std::strcmp(mode, "off") == 0 || p->batch == 0) return;
  const std::string key = tune_key(p);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    tune_load_locked();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      if (p->many) {
        p->tuned_clusters = it->second.first & 0xffff;
        p->long_twopass = (it->second.first >> 16) & 1;
        p->fs_h16 = p->kind == 1 ? (it->second.first >> 17) & 1 : 0;
        p->per_length = (it->second.first >> 18) & 1;
      } else {
        p->variant = it->second.first;
      }
      return;
    }
  }
  if (std::strcmp(mode, "full") == 0) {
    int chosen = 0;
    bfpfft_plan_tune(p, 0, &chosen, nullptr);
  }
}

}  // namespace

extern "C" {

int bfpfft_version(void) { return 100; }

const char* bfpfft_error_string(int status) {
  switch (status) {
    case BFPFFT_OK: return "ok";
    case BFPFFT_ERR_INVALID_ARG: return "invalid argument";
    case BFPFFT_ERR_UNSUPPORTED: return "unsupported length, dtype or direction";
    case BFPFFT_ERR_CUDA: return "CUDA runtime error";
    case BFPFFT_ERR_OOM: return "device out of memory";
    case BFPFFT_ERR_TIMEOUT: return "device-side wait timed out";
    case BFPFFT_ERR_NONFINITE: return "output holds Inf or NaN";
    case BFPFFT_ERR_MISALIGNED: return "buffer not 16-byte aligned";
    default: return "unknown status";
  }
}

int bfpfft_plan_create(bfpfft_plan* out, int64_t n, int64_t batch, int dtype, int direction) {
  if (out == nullptr) return BFPFFT_ERR_INVALID_ARG;
  *out = nullptr;
  if (batch < 0 || !valid_dtype(dtype)) return BFPFFT_ERR_INVALID_ARG;
  if (direction != BFPFFT_FORWARD && direction != BFPFFT_INVERSE) return BFPFFT_ERR_INVALID_ARG;
  const int l = log2_exact(n);
  if (l < kMinLog2 || l > kMaxLog2) return BFPFFT_ERR_UNSUPPORTED;
  if (dtype == BFPFFT_F16_ADAPTIVE && l > bfp::kAdaptiveMaxLog2) return BFPFFT_ERR_UNSUPPORTED;
  if (dtype == BFPFFT_BF16 && l > bfp::kRows16MaxLog2) return BFPFFT_ERR_UNSUPPORTED;
  if (fault("plan")) return BFPFFT_ERR_CUDA;
  if (fault("alloc")) return BFPFFT_ERR_OOM;
  bfpfft_plan p = new (std::nothrow) bfpfft_plan_s();
  if (p == nullptr) return BFPFFT_ERR_OOM;
  p->n = n;
  p->batch = batch;
  p->log2n = l;
  p->dtype = dtype;
  p->direction = direction;
  p->in_exp = 0;
  p->out_exp = 0;
  p->arith = dtype == BFPFFT_BF16 ? BFPFFT_ARITH_BF16 : BFPFFT_ARITH_F32;
  if (dtype == BFPFFT_E4M3_BFP || dtype == BFPFFT_E5M2_BFP) {
    const int s = (l + 1) / 2;            // ceil(log2(n) / 2)
    if (direction == BFPFFT_FORWARD) p->out_exp = s; else p->in_exp = s;
  }
  cudaError_t e = cudaGetDevice(&p->device);
  int st = e == cudaSuccess ? get_twiddles(l, &p->tw) : cuda_status(e);
  if (st == BFPFFT_OK) st = alloc_plan_status(&p->status);
  if (st != BFPFFT_OK) {
    free_plan_resources(p);
    delete p;
    return st;
  }
  tune_on_create(p);
  *out = p;
  return BFPFFT_OK;
}

int bfpfft_plan_create_many(bfpfft_plan* out, int64_t count, const int64_t* n, const int64_t* offset_pts,
                            int dtype, int direction) {
  if (out == nullptr) return BFPFFT_ERR_INVALID_ARG;
  *out = nullptr;
  if (count < 0 || (count > 0 && (n == nullptr || offset_pts == nullptr))) return BFPFFT_ERR_INVALID_ARG;
  if (!valid_dtype(dtype)) return BFPFFT_ERR_INVALID_ARG;
  if (direction != BFPFFT_FORWARD && direction != BFPFFT_INVERSE) return BFPFFT_ERR_INVALID_ARG;
  const int kind = uneven_kind(dtype);
  if (kind < 0) return BFPFFT_ERR_UNSUPPORTED;
  if (count > (int64_t(1) << 30)) return BFPFFT_ERR_UNSUPPORTED;
  // Group line indices by length class, largest first, input order within a class.
  std::vector<std::vector<int64_t>> by_class(kMaxLog2 + 1);
  for (int64_t i = 0; i < count; ++i) {
    const int l = log2_exact(n[i]);
    if (l < kMinLog2 || l > kMaxLog2) return BFPFFT_ERR_UNSUPPORTED;
    if (offset_pts[i] < 0 || offset_pts[i] % 16 != 0) return BFPFFT_ERR_INVALID_ARG;
    by_class[l].push_back(i);
  }
  if (fault("plan")) return BFPFFT_ERR_CUDA;
  if (fault("alloc")) return BFPFFT_ERR_OOM;
  std::vector<long long> line_off;
  std::vector<bfp::UnevenTask> tasks;
  line_off.reserve(size_t(count));
  for (int l = kMaxLog2; l >= kMinLog2; --l) {
    const auto& idx = by_class[l];
    if (idx.empty()) continue;
    const int per_task = bfp::kUnevenTaskPoints >> l;
    for (size_t i = 0; i < idx.size(); i += size_t(per_task)) {
      bfp::UnevenTask t{};
      t.log2n = l;
      t.first = int(line_off.size() + 0);
      t.count = int(std::min<size_t>(size_t(per_task), idx.size() - i));
      for (int k = 0; k < t.count; ++k) line_off.push_back(offset_pts[idx[i + size_t(k)]]);
      tasks.push_back(t);
    }
  }
  bfpfft_plan p = new (std::nothrow) bfpfft_plan_s();
  if (p == nullptr) return BFPFFT_ERR_OOM;
  p->n = 0;
  p->batch = count;
  p->log2n = 0;
  p->dtype = dtype;
  p->direction = direction;
  p->in_exp = p->out_exp = 0;
  p->many = true;
  p->kind = kind;
  p->num_tasks = int(tasks.size());
  // Tasks are sorted longest first: lines of 65536 and 32768 points come first.
  p->first_short_task = 0;
  for (const auto& t : tasks) {
    if (t.log2n >= 13) p->has_fourstep = 1;
    if (p->len_count[t.log2n] == 0) p->len_first[t.log2n] = t.first;
    p->len_count[t.log2n] += t.count;
  }
  for (const auto& t : tasks) {
    if (t.log2n < 15) break;
    ++p->first_short_task;
    const int c = 16 - t.log2n;
    if (p->long_count[c] == 0) p->long_first[c] = t.first;
    p->long_count[c] += t.count;
  }
  int st = BFPFFT_OK;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) st = cuda_status(e);
  if (st == BFPFFT_OK) st = alloc_plan_status(&p->status);
  const float2* tw_host[kMaxLog2 + 1] = {};
  const float2* tw4_host[kMaxLog2 + 1] = {};
  for (int l = kMinLog2; l <= kMaxLog2 && st == BFPFFT_OK; ++l) {
    if (by_class[l].empty()) continue;
    float2* t = nullptr;
    st = get_twiddles(l, &t);
    tw_host[l] = t;
    p->tw_len[l] = t;
    if (st == BFPFFT_OK && l >= 13) {
      bfp::RowArgs tmp{};
      st = fourstep_tables(l, &tmp);
      tw_host[12] = tmp.tw_line;
      tw4_host[l] = tmp.tw_4step;
    }
  }
  if (st == BFPFFT_OK && count > 0) {
    e = cudaMalloc(&p->d_line_off, sizeof(long long) * line_off.size());
    if (e == cudaSuccess) e = cudaMalloc(&p->d_tasks, sizeof(bfp::UnevenTask) * tasks.size());
    if (e == cudaSuccess) e = cudaMalloc(&p->d_tw, sizeof(tw_host));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_tw4, sizeof(tw4_host));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_counter, sizeof(int));
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_line_off, line_off.data(), sizeof(long long) * line_off.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_tasks, tasks.data(), sizeof(bfp::UnevenTask) * tasks.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_tw, tw_host, sizeof(tw_host), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_tw4, tw4_host, sizeof(tw4_host), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = bfp::uneven_max_clusters(kind, direction == BFPFFT_INVERSE, &p->clusters);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) st = cuda_status(e);
    if (st == BFPFFT_OK && p->clusters <= 0) st = BFPFFT_ERR_UNSUPPORTED;
  }
  if (st != BFPFFT_OK) {
    free_plan_resources(p);
    delete p;
    return st;
  }
  tune_on_create(p);
  *out = p;
  return BFPFFT_OK;
}

int bfpfft_plan_info(bfpfft_plan plan, int64_t* tasks, int64_t* clusters) {
  if (plan == nullptr || tasks == nullptr || clusters == nullptr) return BFPFFT_ERR_INVALID_ARG;
  *tasks = plan->many ? plan->num_tasks : 0;
  *clusters = plan->many ? plan->clusters : 0;
  return BFPFFT_OK;
}


int bfpfft_exec(bfpfft_plan plan, const void* in, void* out, void* stream) {
  if (plan == nullptr) return BFPFFT_ERR_INVALID_ARG;
  if (plan->batch == 0) return BFPFFT_OK;
  if (plan->many) {
    if (in == nullptr || out == nullptr) return BFPFFT_ERR_INVALID_ARG;
    if (!aligned16(in) || !aligned16(out)) return BFPFFT_ERR_MISALIGNED;
    if (fault("launch")) return BFPFFT_ERR_CUDA;
    return exec_many(plan, in, out, static_cast<cudaStream_t>(stream));
  }
  if (in == nullptr || out == nullptr) return BFPFFT_ERR_INVALID_ARG;
  if (plan->dtype == BFPFFT_F16_ADAPTIVE) return BFPFFT_ERR_INVALID_ARG;   // needs bfpfft_exec_adaptive
  if (!aligned16(in) || !aligned16(out)) return BFPFFT_ERR_MISALIGNED;
  if (fault("launch")) return BFPFFT_ERR_CUDA;
  bfp::RowArgs a{};
  a.in = in;
  a.out = out;
  a.tw = plan->tw;
  a.h = nullptr;
  a.status = plan->status;
  a.finite_flag = (plan->flags & BFPFFT_CHECK_FINITE) ? plan->status : nullptr;
  a.variant = std::getenv("BFPFFT_ROWS") == nullptr && plan->variant >= 0 ? plan->variant : rows_variant();
  if (!device_memory(in)) {
    a.variant = without_l2(a.variant);
    a.no_prefetch = 1;
  }
  a.fs_h16 = plan->dtype == BFPFFT_F16_BFP && fp16_exchange_variant(a.variant);
  if (plan->log2n >= 15 && a.variant == bfp::kRowsTwoPass && plan->dtype != BFPFFT_F16_NAIVE &&
      plan->dtype != BFPFFT_BF16 && plan->dtype != BFPFFT_F16_ADAPTIVE) {
    return run_twopass(uneven_kind(plan->dtype), plan->log2n,
                       plan->direction == BFPFFT_FORWARD ? bfp::kForward : bfp::kInverse, in, out, nullptr,
                       plan->batch, std::ldexp(1.0f, plan->in_exp), std::ldexp(1.0f, -plan->out_exp),
                       a.finite_flag, static_cast<cudaStream_t>(stream));
  }
  if (plan->arith == BFPFFT_ARITH_F16_MUL_F32_ACC) a.variant = bfp::kRowsTc;
  if (plan->arith == BFPFFT_ARITH_F16 || plan->arith == BFPFFT_ARITH_BF16) {
    const bool bf16 = plan->arith == BFPFFT_ARITH_BF16;
    const int st16 = get_twiddles16(plan->log2n, bf16, &a.tw16);
    if (st16 != BFPFFT_OK) return st16;
    a.lines = plan->batch;
    a.in_stride = plan->n;
    a.out_stride = plan->n;
    a.no_prefetch = device_memory(in) ? 0 : 1;
    const int mode16 = plan->direction == BFPFFT_FORWARD ? bfp::kForward : bfp::kInverse;
    cudaStream_t s16 = static_cast<cudaStream_t>(stream);
    return cuda_status(bf16 ? bfp::launch_rows16_bf16(plan->log2n, mode16, a, s16)
                            : bfp::launch_rows16_f16(plan->log2n, mode16, plan->dtype == BFPFFT_F16_NAIVE, a, s16));
  }
  if (a.variant == bfp::kRowsTc && plan->log2n == 12 &&
      (plan->dtype == BFPFFT_F16_BFP || plan->dtype == BFPFFT_E4M3_BFP || plan->dtype == BFPFFT_E5M2_BFP)) {
    const int stc = get_tc_matrix(const_cast<void**>(&a.tc_b));
    if (stc != BFPFFT_OK) return stc;
  }
  {
    const int st4 = fourstep_tables(plan->log2n, &a);
    if (st4 != BFPFFT_OK) return st4;
  }
  a.lines = plan->batch;
  a.in_stride = plan->n;
  a.out_stride = plan->n;
  a.in_scale = std::ldexp(1.0f, plan->in_exp);
  a.out_scale = std::ldexp(1.0f, -plan->out_exp);
  const int mode = plan->direction == BFPFFT_FORWARD ? bfp::kForward : bfp::kInverse;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  switch (plan->dtype) {
    case BFPFFT_F32: e = bfp::launch_rows_f32(plan->log2n, mode, a, s); break;
    case BFPFFT_F16_BFP: e = bfp::launch_rows_f16(plan->log2n, mode, false, a, s); break;
    case BFPFFT_F16_NAIVE: e = bfp::launch_rows_f16(plan->log2n, mode, true, a, s); break;
    case BFPFFT_E4M3_BFP:
    case BFPFFT_E5M2_BFP: {
      const int fmt = plan->dtype == BFPFFT_E4M3_BFP ? 0 : 1;
      e = plan->arith == BFPFFT_ARITH_F16_MUL_F32_ACC ? bfp::launch_tc_fp8(mode, fmt, a, s)
                                                      : bfp::launch_rows_fp8(plan->log2n, mode, fmt, a, s);
      break;
    }
    default: return BFPFFT_ERR_UNSUPPORTED;
  }
  return cuda_status(e);
}

int bfpfft_plan_destroy(bfpfft_plan plan) {
  if (plan == nullptr) return BFPFFT_OK;
  if (plan->many || plan->graph) cudaDeviceSynchronize();
  free_plan_resources(plan);
  delete plan;
  return BFPFFT_OK;
}

int bfpfft_exec_graph(bfpfft_plan plan, const void* in, void* out, void* stream) {
  if (plan == nullptr) return BFPFFT_ERR_INVALID_ARG;
  if (plan->batch == 0) return BFPFFT_OK;
  if (in == nullptr || out == nullptr) return BFPFFT_ERR_INVALID_ARG;
  if (!aligned16(in) || !aligned16(out)) return BFPFFT_ERR_MISALIGNED;
  if (plan->graph == nullptr || plan->graph_in != in || plan->graph_out != out) {
    if (plan->graph) {
      cudaGraphExecDestroy(plan->graph);
      plan->graph = nullptr;
    }
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    int st = BFPFFT_OK;
    if (e == cudaSuccess) st = bfpfft_exec(plan, in, out, cap);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && st == BFPFFT_OK) e = cudaGraphInstantiate(&plan->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (st != BFPFFT_OK) return st;
    if (e != cudaSuccess) {
      plan->graph = nullptr;
      return cuda_status(e);
    }
    plan->graph_in = in;
    plan->graph_out = out;
  }
  return cuda_status(cudaGraphLaunch(plan->graph, static_cast<cudaStream_t>(stream)));
}

int bfpfft_plan_scale_exp(bfpfft_plan plan, int* in_exp, int* out_exp) {
  if (plan == nullptr || in_exp == nullptr || out_exp == nullptr) return BFPFFT_ERR_INVALID_ARG;
  *in_exp = plan->in_exp;
  *out_exp = plan->out_exp;
  return BFPFFT_OK;
}

int bfpfft_device_status(int* status) {
  if (status == nullptr) return BFPFFT_ERR_INVALID_ARG;
  int* w = nullptr;
  int st = get_status_word(&w);
  if (st != BFPFFT_OK) return st;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(status, w, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(w, 0, sizeof(int));
  return cuda_status(e);
}

int bfpfft_plan_status(bfpfft_plan plan, int* status) {
  if (plan == nullptr || status == nullptr) return BFPFFT_ERR_INVALID_ARG;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(status, plan->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(plan->status, 0, sizeof(int));
  return cuda_status(e);
}

int bfpfft_plan_set_many_schedule(bfpfft_plan plan, int clusters, int flags) {
  if (plan == nullptr || !plan->many || clusters < 0) return BFPFFT_ERR_INVALID_ARG;
  if ((flags & ~(BFPFFT_MANY_TWO_PASS | BFPFFT_MANY_FP16_ROWS | BFPFFT_MANY_PER_LENGTH)) != 0)
    return BFPFFT_ERR_INVALID_ARG;
  if ((flags & BFPFFT_MANY_FP16_ROWS) && plan->kind != 1) return BFPFFT_ERR_INVALID_ARG;
  plan->tuned_clusters = std::min(clusters, plan->clusters);
  plan->long_twopass = (flags & BFPFFT_MANY_TWO_PASS) ? 1 : 0;
  plan->fs_h16 = (flags & BFPFFT_MANY_FP16_ROWS) ? 1 : 0;
  plan->per_length = (flags & BFPFFT_MANY_PER_LENGTH) ? 1 : 0;
  if (plan->graph) {
    cudaGraphExecDestroy(plan->graph);
    plan->graph = nullptr;
  }
  return BFPFFT_OK;
}

int bfpfft_plan_set_flags(bfpfft_plan plan, int flags) {
  if (plan == nullptr || (flags & ~BFPFFT_CHECK_FINITE) != 0) return BFPFFT_ERR_INVALID_ARG;
  plan->flags = flags;
  if (plan->graph) {   // a captured graph holds the old flags: capture again on the next call
    cudaGraphExecDestroy(plan->graph);
    plan->graph = nullptr;
  }
  return BFPFFT_OK;
}

int bfpfft_plan_set_arith(bfpfft_plan plan, int arith) {
  if (plan == nullptr) return BFPFFT_ERR_INVALID_ARG;
  if (arith < BFPFFT_ARITH_F32 || arith > BFPFFT_ARITH_BF16) return BFPFFT_ERR_INVALID_ARG;
  const bool f16 = plan->dtype == BFPFFT_F16_BFP || plan->dtype == BFPFFT_F16_NAIVE;
  bool ok = false;
  switch (arith) {
    case BFPFFT_ARITH_F32: ok = plan->dtype != BFPFFT_BF16; break;
    case BFPFFT_ARITH_F16: ok = !plan->many && f16 && plan->log2n <= bfp::kRows16MaxLog2; break;
    case BFPFFT_ARITH_F16_MUL_F32_ACC:
      ok = !plan->many && plan->log2n == 12 &&
           (plan->dtype == BFPFFT_F16_BFP || plan->dtype == BFPFFT_E4M3_BFP || plan->dtype == BFPFFT_E5M2_BFP);
      break;
    case BFPFFT_ARITH_BF16: ok = plan->dtype == BFPFFT_BF16; break;
    default: break;
  }
  if (!ok) return BFPFFT_ERR_UNSUPPORTED;
  if (arith == BFPFFT_ARITH_F16 || arith == BFPFFT_ARITH_BF16) {   // the table now, not inside a capture
    const void* tw16 = nullptr;
    const int st = get_twiddles16(plan->log2n, arith == BFPFFT_ARITH_BF16, &tw16);
    if (st != BFPFFT_OK) return st;
  }
  plan->arith = arith;
  if (plan->graph) {
    cudaGraphExecDestroy(plan->graph);
    plan->graph = nullptr;
  }
  return BFPFFT_OK;
}

int bfpfft_plan_selftest_wait(bfpfft_plan plan, void* stream) {
  if (plan == nullptr) return BFPFFT_ERR_INVALID_ARG;
  if (fault("launch")) return BFPFFT_ERR_CUDA;
  wait_selftest_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(plan->status);
  return cuda_status(cudaGetLastError());
}

int bfpfft_exec_adaptive(bfpfft_plan plan, const void* in, const int32_t* in_exp, void* out, int32_t* out_exp,
                         void* stream) {
  if (plan == nullptr || in == nullptr || out == nullptr || out_exp == nullptr) return BFPFFT_ERR_INVALID_ARG;
  if (plan->dtype != BFPFFT_F16_ADAPTIVE) return BFPFFT_ERR_INVALID_ARG;
  if (plan->batch == 0) return BFPFFT_OK;
  if (!aligned16(in) || !aligned16(out)) return BFPFFT_ERR_MISALIGNED;
  if (fault("launch")) return BFPFFT_ERR_CUDA;
  bfp::RowArgs a{};
  a.in = in;
  a.out = out;
  a.tw = plan->tw;
  a.status = plan->status;
  a.finite_flag = (plan->flags & BFPFFT_CHECK_FINITE) ? plan->status : nullptr;
  a.no_prefetch = device_memory(in) ? 0 : 1;
  a.lines = plan->batch;
  a.in_stride = plan->n;
  a.out_stride = plan->n;
  a.in_scale = a.out_scale = 1.f;
  a.in_exp = in_exp;
  a.out_exp = out_exp;
  const int mode = plan->direction == BFPFFT_FORWARD ? bfp::kForward : bfp::kInverse;
  return cuda_status(bfp::launch_rows_adaptive_f16(plan->log2n, mode, a, static_cast<cudaStream_t>(stream)));
}

int bfp_spectral_adaptive(const void* x, int x_dtype, const int32_t* x_exp, const void* h, void* out,
                          int32_t* out_exp, int64_t n, int64_t lines, void* stream) {
  if (lines < 0) return BFPFFT_ERR_INVALID_ARG;
  const int l = log2_exact(n);
  if (l < kMinLog2 || l > bfp::kAdaptiveMaxLog2) return BFPFFT_ERR_UNSUPPORTED;
  if (x_dtype != BFPFFT_F32 && x_dtype != BFPFFT_F16_ADAPTIVE) return BFPFFT_ERR_UNSUPPORTED;
  if (x_dtype == BFPFFT_F32 && x_exp != nullptr) return BFPFFT_ERR_INVALID_ARG;
  if (lines == 0) return BFPFFT_OK;
  if (x == nullptr || h == nullptr || out == nullptr || out_exp == nullptr) return BFPFFT_ERR_INVALID_ARG;
  if (!aligned16(x) || !aligned16(h) || !aligned16(out)) return BFPFFT_ERR_MISALIGNED;
  if (fault("launch")) return BFPFFT_ERR_CUDA;
  bfp::RowArgs a;
  int st = row_args(l, &a);
  if (st != BFPFFT_OK) return st;
  a.in = x;
  a.out = out;
  a.h = static_cast<const float2*>(h);
  a.no_prefetch = device_memory(x) ? 0 : 1;
  a.lines = lines;
  a.in_stride = n;
  a.out_stride = n;
  a.in_exp = x_exp;
  a.out_exp = out_exp;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cudaError_t e = x_dtype == BFPFFT_F32 ? bfp::launch_spectral_adaptive_c64(l, a, s)
                                              : bfp::launch_rows_adaptive_f16(l, bfp::kCompress, a, s);
  return cuda_status(e);
}

static int sar_arith_check(int arith, int l, int in_dtype, int out_dtype, bool azimuth);
static cudaError_t sar_lines(int l, int arith, bool in16, bool out16, bool naive, bool tload, bool tstore,
                             const bfp::RowArgs& a, cudaStream_t s);

int bfp_spectral_filter(const void* x, int x_dtype, const void* h, int64_t h_stride, void* out, int out_dtype,
                        int64_t n, int64_t lines, int arith, void* stream) {
  if (lines < 0) return BFPFFT_ERR_INVALID_ARG;
  if (arith != BFPFFT_ARITH_F32 && arith != BFPFFT_ARITH_F16 && arith != BFPFFT_ARITH_F16_MUL_F32_ACC)
    return BFPFFT_ERR_INVALID_ARG;
  if (h_stride != 0 && h_stride != n) return BFPFFT_ERR_INVALID_ARG;
  const int l = log2_exact(n);
  if (l < bfp::kSarMinLog2 || l > kSarMaxLog2) return BFPFFT_ERR_UNSUPPORTED;
  if (x_dtype != BFPFFT_F32 && x_dtype != BFPFFT_F16_BFP) return BFPFFT_ERR_UNSUPPORTED;
  if (out_dtype != BFPFFT_F32 && out_dtype != BFPFFT_F16_BFP && out_dtype != BFPFFT_F16_NAIVE)
    return BFPFFT_ERR_UNSUPPORTED;
  if (const int ac = sar_arith_check(arith, l, x_dtype, out_dtype, false); ac != BFPFFT_OK) return ac;
  if (lines == 0) return BFPFFT_OK;
  if (x == nullptr || h == nullptr || out == nullptr) return BFPFFT_ERR_INVALID_ARG;
  if (!aligned16(x) || !aligned16(h) || !aligned16(out)) return BFPFFT_ERR_MISALIGNED;
  if (fault("launch")) return BFPFFT_ERR_CUDA;
  bfp::RowArgs a;
  int st = row_args(l, &a);
  if (st != BFPFFT_OK) return st;
  if (arith == BFPFFT_ARITH_F16 && (st = get_twiddles16(l, false, &a.tw16)) != BFPFFT_OK) return st;
  if (arith == BFPFFT_ARITH_F16_MUL_F32_ACC && (st = get_tc_matrix(const_cast<void**>(&a.tc_b))) != BFPFFT_OK)
    return st;
  a.in = x;
  a.out = out;
  a.h = static_cast<const float2*>(h);
  a.h_stride = h_stride;
  if (!device_memory(x)) {
    a.variant = without_l2(a.variant);
    a.no_prefetch = 1;
  }
  a.lines = lines;
  a.in_stride = n;
  a.out_stride = n;
  const bool naive = out_dtype == BFPFFT_F16_NAIVE;
  return cuda_status(sar_lines(l, arith, x_dtype == BFPFFT_F16_BFP, out_dtype != BFPFFT_F32, naive, false, false, a,
                               static_cast<cudaStream_t>(stream)));
}

int sar_make_filter(const void* ref, int64_t n, int peak_normalise, void* h_out, void* stream) {
  if (ref == nullptr || h_out == nullptr) return BFPFFT_ERR_INVALID_ARG;
  if (!aligned16(ref) || !aligned16(h_out)) return BFPFFT_ERR_MISALIGNED;
  const int l = log2_exact(n);
  if (l < kMinLog2 || l > kMaxLog2) return BFPFFT_ERR_UNSUPPORTED;
  if (fault("launch")) return BFPFFT_ERR_CUDA;
  bfp::RowArgs a;
  int st = row_args(l, &a);
  if (st != BFPFFT_OK) return st;
  a.in = ref;
  a.out = h_out;
  a.lines = 1;
  a.in_stride = n;
  a.out_stride = n;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = bfp::launch_rows_f32(l, bfp::kForward, a, s);
  if (e != cudaSuccess) return cuda_status(e);
  conj_normalise_kernel<<<1, 1024, 0, s>>>(static_cast<float2*>(h_out), int(n), peak_normalise);
  return cuda_status(cudaGetLastError());
}


int sar_range_compress(const void* raw, int raw_dtype, void* out, int out_dtype, const void* hr,
                       int64_t n_az, int64_t n_rg, int transpose_out, void* stream) {
  return sar_range_compress_arith(raw, raw_dtype, out, out_dtype, hr, n_az, n_rg, transpose_out, BFPFFT_ARITH_F32,
                                  stream);
}

// The compression lines of a SAR call: the FP32-arithmetic kernels; with
// BFPFFT_ARITH_F16 the FP16-arithmetic kernel; with
// BFPFFT_ARITH_F16_MUL_F32_ACC the tensor-core kernel (N = 4096).  The last
// two write dense FP16 rows.
static cudaError_t sar_lines(int l, int arith, bool in16, bool out16, bool naive, bool tload, bool tstore,
                             const bfp::RowArgs& a, cudaStream_t s) {
  if (arith == BFPFFT_ARITH_F16) return bfp::launch_rows16_compress_f16(l, !in16, naive, a, s);
  if (arith == BFPFFT_ARITH_F16_MUL_F32_ACC) return bfp::launch_tc_compress(!in16, a, s);
  return bfp::launch_sar(l, in16, out16, naive, tload, tstore, a, s);
}

// Arguments a SAR call's arithmetic mode accepts: FP16 arithmetic writes FP16
// (BFP or naive); the tensor-core lines take N = 4096 and write FP16-BFP.
static int sar_arith_check(int arith, int l, int in_dtype, int out_dtype, bool azimuth) {
  if (arith != BFPFFT_ARITH_F32 && arith != BFPFFT_ARITH_F16 && arith != BFPFFT_ARITH_F16_MUL_F32_ACC)
    return BFPFFT_ERR_INVALID_ARG;
  if (arith == BFPFFT_ARITH_F16 && (out_dtype == BFPFFT_F32 || (azimuth && in_dtype != BFPFFT_F16_BFP)))
    return BFPFFT_ERR_UNSUPPORTED;
  if (arith == BFPFFT_ARITH_F16_MUL_F32_ACC && (l != 12 || out_dtype != BFPFFT_F16_BFP))
    return BFPFFT_ERR_UNSUPPORTED;
  return BFPFFT_OK;
}

int sar_range_compress_arith(const void* raw, int raw_dtype, void* out, int out_dtype, const void* hr,
                             int64_t n_az, int64_t n_rg, int transpose_out, int arith, void* stream) {
  if (n_az < 0) return BFPFFT_ERR_INVALID_ARG;
  if (arith != BFPFFT_ARITH_F32 && arith != BFPFFT_ARITH_F16 && arith != BFPFFT_ARITH_F16_MUL_F32_ACC)
    return BFPFFT_ERR_INVALID_ARG;
  const int l = log2_exact(n_rg);
  if (l < bfp::kSarMinLog2 || l > kSarMaxLog2) return BFPFFT_ERR_UNSUPPORTED;
  if (n_az == 0) return BFPFFT_OK;
  if (raw == nullptr || out == nullptr || hr == nullptr) return BFPFFT_ERR_INVALID_ARG;
  if (!aligned16(raw) || !aligned16(out) || !aligned16(hr)) return BFPFFT_ERR_MISALIGNED;
  if (raw_dtype != BFPFFT_F32 && raw_dtype != BFPFFT_F16_BFP) return BFPFFT_ERR_UNSUPPORTED;
  if (out_dtype != BFPFFT_F32 && out_dtype != BFPFFT_F16_BFP && out_dtype != BFPFFT_F16_NAIVE)
    return BFPFFT_ERR_UNSUPPORTED;
  if (const int ac = sar_arith_check(arith, l, raw_dtype, out_dtype, false); ac != BFPFFT_OK) return ac;
  if (transpose_out != 0 && transpose_out != 1) return BFPFFT_ERR_INVALID_ARG;
  if (fault("launch")) return BFPFFT_ERR_CUDA;
  bfp::RowArgs a;
  int st = row_args(l, &a);
  if (st != BFPFFT_OK) return st;
  if (arith == BFPFFT_ARITH_F16 && (st = get_twiddles16(l, false, &a.tw16)) != BFPFFT_OK) return st;
  if (arith == BFPFFT_ARITH_F16_MUL_F32_ACC && (st = get_tc_matrix(const_cast<void**>(&a.tc_b))) != BFPFFT_OK)
    return st;
  a.in = raw;
  a.out = out;
  a.h = static_cast<const float2*>(hr);
  if (!device_memory(raw)) {
    a.variant = without_l2(a.variant);
    a.no_prefetch = 1;
  }
  a.lines = n_az;
  a.in_stride = n_rg;
  a.out_stride = transpose_out ? n_az : n_rg;
  const bool naive = out_dtype == BFPFFT_F16_NAIVE;
  const bool in16 = raw_dtype == BFPFFT_F16_BFP;
  const bool out16 = out_dtype != BFPFFT_F32;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (transpose_out && (sar_split_turns() || arith != BFPFFT_ARITH_F32)) {
    // Rows into scratch [n_az][n_rg], then turned into out [n_rg][n_az].
    const int eb = out16 ? 4 : 8;
    void* tmp = nullptr;
    cudaError_t e = scratch_alloc(&tmp, size_t(n_az) * size_t(n_rg) * eb, s);
    if (e != cudaSuccess) return cuda_status(e);
    a.out = tmp;
    a.out_stride = n_rg;
    e = sar_lines(l, arith, in16, out16, naive, false, false, a, s);
    if (e == cudaSuccess) e = bfp::launch_transpose(tmp, out, n_az, n_rg, eb, s);
    const cudaError_t f = cudaFreeAsync(tmp, s);
    return cuda_status(e != cudaSuccess ? e : f);
  }
  cudaError_t e = sar_lines(l, arith, in16, out16, naive, /*tload=*/false, transpose_out != 0, a, s);
  return cuda_status(e);
}

int sar_azimuth_compress(const void* rc, int rc_dtype, int rc_layout, void* img, int img_dtype,
                         const void* ha, int64_t n_az, int64_t n_rg, void* stream) {
  return sar_azimuth_compress_arith(rc, rc_dtype, rc_layout, img, img_dtype, ha, n_az, n_rg, BFPFFT_ARITH_F32,
                                    stream);
}

int sar_azimuth_compress_arith(const void* rc, int rc_dtype, int rc_layout, void* img, int img_dtype,
                               const void* ha, int64_t n_az, int64_t n_rg, int arith, void* stream) {
  if (n_rg < 0) return BFPFFT_ERR_INVALID_ARG;
  if (arith != BFPFFT_ARITH_F32 && arith != BFPFFT_ARITH_F16 && arith != BFPFFT_ARITH_F16_MUL_F32_ACC)
    return BFPFFT_ERR_INVALID_ARG;
  const int l = log2_exact(n_az);
  if (l < bfp::kSarMinLog2 || l > kSarMaxLog2) return BFPFFT_ERR_UNSUPPORTED;
  if (n_rg == 0) return BFPFFT_OK;
  if (rc == nullptr || img == nullptr || ha == nullptr) return BFPFFT_ERR_INVALID_ARG;
  if (!aligned16(rc) || !aligned16(img) || !aligned16(ha)) return BFPFFT_ERR_MISALIGNED;
  if (rc_dtype != BFPFFT_F32 && rc_dtype != BFPFFT_F16_BFP) return BFPFFT_ERR_UNSUPPORTED;
  if (img_dtype != BFPFFT_F32 && img_dtype != BFPFFT_F16_BFP && img_dtype != BFPFFT_F16_NAIVE)
    return BFPFFT_ERR_UNSUPPORTED;
  if (const int ac = sar_arith_check(arith, l, rc_dtype, img_dtype, true); ac != BFPFFT_OK) return ac;
  if (rc_layout != 0 && rc_layout != 1) return BFPFFT_ERR_INVALID_ARG;
  if (fault("launch")) return BFPFFT_ERR_CUDA;
  bfp::RowArgs a;
  int st = row_args(l, &a);
  if (st != BFPFFT_OK) return st;
  if (arith == BFPFFT_ARITH_F16 && (st = get_twiddles16(l, false, &a.tw16)) != BFPFFT_OK) return st;
  if (arith == BFPFFT_ARITH_F16_MUL_F32_ACC && (st = get_tc_matrix(const_cast<void**>(&a.tc_b))) != BFPFFT_OK)
    return st;
  a.in = rc;
  a.out = img;
  a.h = static_cast<const float2*>(ha);
  if (!device_memory(rc)) {
    a.variant = without_l2(a.variant);
    a.no_prefetch = 1;
  }
  a.lines = n_rg;                                   // one line per range column
  a.in_stride = rc_layout == 0 ? n_rg : n_az;       // [n_az][n_rg] column vs [n_rg][n_az] row
  a.out_stride = n_rg;                              // image is [n_az][n_rg]
  const bool naive = img_dtype == BFPFFT_F16_NAIVE;
  const bool in16 = rc_dtype == BFPFFT_F16_BFP, out16 = img_dtype != BFPFFT_F32;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (sar_split_turns() || arith != BFPFFT_ARITH_F32) {
    // Layout 0 is first turned to [n_rg][n_az]; the azimuth lines are then
    // dense rows, compressed into scratch and turned into img [n_az][n_rg].
    const size_t pts = size_t(n_az) * size_t(n_rg);
    const int ib = in16 ? 4 : 8, ob = out16 ? 4 : 8;
    void* rows_in = nullptr;
    void* rows_out = nullptr;
    cudaError_t e = cudaSuccess;
    if (rc_layout == 0) e = scratch_alloc(&rows_in, pts * ib, s);
    if (e == cudaSuccess) e = scratch_alloc(&rows_out, pts * ob, s);
    if (e == cudaSuccess && rc_layout == 0) e = bfp::launch_transpose(rc, rows_in, n_az, n_rg, ib, s);
    if (e == cudaSuccess) {
      a.in = rc_layout == 0 ? rows_in : rc;
      a.in_stride = n_az;
      a.out = rows_out;
      a.out_stride = n_az;
      e = sar_lines(l, arith, in16, out16, naive, false, false, a, s);
    }
    if (e == cudaSuccess) e = bfp::launch_transpose(rows_out, img, n_rg, n_az, ob, s);
    cudaError_t f = cudaSuccess;
    if (rows_out != nullptr) f = cudaFreeAsync(rows_out, s);
    if (rows_in != nullptr && f == cudaSuccess) f = cudaFreeAsync(rows_in, s);
    return cuda_status(e != cudaSuccess ? e : f);
  }
  cudaError_t e = bfp::launch_sar(l, in16, out16, naive, /*tload=*/rc_layout == 0, /*tstore=*/true, a, s);
  return cuda_status(e);
}

int sar_rda_image(const void* raw, int raw_dtype, void* img, int img_dtype, const void* hr, int64_t n_az,
                  int64_t n_rg, const double* geometry, int64_t aperture, int flags, void* stream) {
  if (n_az < 0 || n_rg < 0) return BFPFFT_ERR_INVALID_ARG;
  const int la = log2_exact(n_az), lr = log2_exact(n_rg);
  if (la < bfp::kRdaMinLog2 || la > bfp::kRdaMaxLog2 || lr < bfp::kRdaMinLog2 || lr > bfp::kRdaMaxLog2)
    return BFPFFT_ERR_UNSUPPORTED;
  if (raw_dtype != BFPFFT_F32 && raw_dtype != BFPFFT_F16_BFP) return BFPFFT_ERR_UNSUPPORTED;
  if (img_dtype != BFPFFT_F32 && img_dtype != BFPFFT_F16_BFP) return BFPFFT_ERR_UNSUPPORTED;
  if ((flags & ~(SAR_RDA_RCMC | SAR_RDA_RANGE_DEPENDENT | SAR_RDA_PEAK_NORMALISE)) != 0) return BFPFFT_ERR_INVALID_ARG;
  if (img_dtype == BFPFFT_F16_BFP && !(flags & SAR_RDA_PEAK_NORMALISE)) return BFPFFT_ERR_UNSUPPORTED;
  if (geometry == nullptr || aperture < 2 || aperture > n_az || (aperture & 1)) return BFPFFT_ERR_INVALID_ARG;
  bfp::RdaGeometry geo{geometry[0], geometry[1], geometry[2], geometry[3], geometry[4]};
  if (!(geo.range_cell_m > 0 && geo.prf_hz > 0 && geo.wavelength_m > 0 && geo.speed_mps > 0 &&
        geo.centre_range_m > 0.5 * double(n_rg) * geo.range_cell_m))
    return BFPFFT_ERR_INVALID_ARG;
  if (geo.wavelength_m * geo.prf_hz / (4.0 * geo.speed_mps) >= 1.0) return BFPFFT_ERR_INVALID_ARG;   // D(f) real
  if (raw == nullptr || img == nullptr || hr == nullptr) return BFPFFT_ERR_INVALID_ARG;
  if (!aligned16(raw) || !aligned16(img) || !aligned16(hr)) return BFPFFT_ERR_MISALIGNED;
  if (fault("launch")) return BFPFFT_ERR_CUDA;
  const bool f16 = img_dtype == BFPFFT_F16_BFP;
  const int eb = f16 ? 4 : 8;
  const size_t bytes = size_t(n_az) * size_t(n_rg) * eb;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bfp::RowArgs ra;
  int st = row_args(lr, &ra);
  if (st != BFPFFT_OK) return st;
  float2* tw_az = nullptr;
  st = get_twiddles(la, &tw_az);
  if (st != BFPFFT_OK) return st;
  void* sa = nullptr;
  void* sb = nullptr;
  cudaError_t e = scratch_alloc(&sa, bytes, s);
  if (e == cudaSuccess) e = scratch_alloc(&sb, bytes, s);
  // 1. range compression: rows of raw into sb [n_az][n_rg], turned into sa [n_rg][n_az]
  if (e == cudaSuccess) {
    ra.in = raw;
    ra.out = sb;
    ra.h = static_cast<const float2*>(hr);
    if (!device_memory(raw)) ra.variant = without_l2(ra.variant);
    ra.lines = n_az;
    ra.in_stride = n_rg;
    ra.out_stride = n_rg;
    e = bfp::launch_sar(lr, raw_dtype == BFPFFT_F16_BFP, f16, false, false, false, ra, s);
  }
  if (e == cudaSuccess) e = bfp::launch_transpose(sb, sa, n_az, n_rg, eb, s);
  // 2. azimuth DFT of every range line, in place: sa holds S[r][f]
  if (e == cudaSuccess) {
    bfp::RowArgs az;
    st = row_args(la, &az);
    if (st != BFPFFT_OK) e = cudaErrorUnknown;
    az.in = sa;
    az.out = sa;
    az.lines = n_rg;
    az.in_stride = n_az;
    az.out_stride = n_az;
    if (e == cudaSuccess)
      e = f16 ? bfp::launch_rows_f16(la, bfp::kForward, false, az, s) : bfp::launch_rows_f32(la, bfp::kForward, az, s);
  }
  bfp::RdaArgs r{};
  r.geo = geo;
  r.aperture = int(aperture);
  r.range_dependent = (flags & SAR_RDA_RANGE_DEPENDENT) ? 1 : 0;
  r.peak_normalise = (flags & SAR_RDA_PEAK_NORMALISE) ? 1 : 0;
  // 3. RCMC along range, one line per Doppler bin ([f][r] layout)
  if (e == cudaSuccess && (flags & SAR_RDA_RCMC)) {
    e = bfp::launch_transpose(sa, sb, n_rg, n_az, eb, s);
    r.in = sb;
    r.out = sb;
    r.tw = ra.tw;
    r.lines = n_az;
    r.other = n_az;
    if (e == cudaSuccess) e = bfp::launch_rcmc_rows(lr, f16, r, s);
    if (e == cudaSuccess) e = bfp::launch_transpose(sb, sa, n_az, n_rg, eb, s);
  }
  // 4. per range bin: its own azimuth filter and the inverse DFT, into sb [n_rg][n_az]
  if (e == cudaSuccess) {
    r.in = sa;
    r.out = sb;
    r.tw = tw_az;
    r.lines = n_rg;
    r.other = n_rg;
    e = bfp::launch_azimuth_rows(la, f16, r, s);
  }
  // 5. turned into the image [n_az][n_rg]
  if (e == cudaSuccess) e = bfp::launch_transpose(sb, img, n_rg, n_az, eb, s);
  cudaError_t f = cudaSuccess;
  if (sb != nullptr) f = cudaFreeAsync(sb, s);
  if (sa != nullptr && f == cudaSuccess) f = cudaFreeAsync(sa, s);
  if (st != BFPFFT_OK) return st;
  return cuda_status(e != cudaSuccess ? e : f);
}

size_t sar_autofocus_workspace_bytes(int64_t n_az) {
  const int l = log2_exact(n_az);
  if (l < bfp::kAfMinLog2 || l > bfp::kAfMaxLog2) return 0;
  return bfp::af_workspace_bytes(n_az);
}

static int autofocus_common(const void* rc, int rc_dtype, const float* phi, const void* ha, int64_t n_az,
                            int64_t n_rg, float* grad_out, void* stats_out, void* workspace, size_t ws_bytes,
                            int arith, void* stream) {
  if (n_rg < 0) return BFPFFT_ERR_INVALID_ARG;
  if (arith != BFPFFT_ARITH_F32 && arith != BFPFFT_ARITH_F16_MUL_F32_ACC) return BFPFFT_ERR_INVALID_ARG;
  const int l = log2_exact(n_az);
  if (l < bfp::kAfMinLog2 || l > bfp::kAfMaxLog2) return BFPFFT_ERR_UNSUPPORTED;
  if (arith == BFPFFT_ARITH_F16_MUL_F32_ACC && l != 12) return BFPFFT_ERR_UNSUPPORTED;
  if (rc_dtype != BFPFFT_F32 && rc_dtype != BFPFFT_F16_BFP) return BFPFFT_ERR_UNSUPPORTED;
  if (rc == nullptr || phi == nullptr || ha == nullptr || stats_out == nullptr || workspace == nullptr)
    return BFPFFT_ERR_INVALID_ARG;
  if (!aligned16(rc) || !aligned16(ha) || !aligned16(stats_out) || !aligned16(workspace) ||
      (grad_out != nullptr && !aligned16(grad_out)))
    return BFPFFT_ERR_MISALIGNED;
  if (ws_bytes < bfp::af_workspace_bytes(n_az)) return BFPFFT_ERR_INVALID_ARG;
  if (fault("launch")) return BFPFFT_ERR_CUDA;
  bfp::RowArgs a;
  int st = row_args(l, &a);
  if (st != BFPFFT_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (arith == BFPFFT_ARITH_F16_MUL_F32_ACC) {
    if ((st = get_tc_matrix(const_cast<void**>(&a.tc_b))) != BFPFFT_OK) return st;
    const bfp::AfWorkspaceLayout wl = bfp::af_workspace_layout(workspace, n_az);
    cudaError_t e = bfp::af_phase_table(phi, wl.ph, n_az, s);
    if (e != cudaSuccess) return cuda_status(e);
    const bfp::AfTcWorkspace tw{wl.sq_part, wl.g_part, wl.q_part, wl.qmax, bfp::kAfMaxCtas};
    e = bfp::launch_autofocus_tc(rc_dtype == BFPFFT_F16_BFP, rc, wl.ph, static_cast<const float2*>(ha), a, n_rg,
                                 static_cast<double*>(stats_out), grad_out, tw, device_memory(rc), s);
    return cuda_status(e);
  }
  cudaError_t e = bfp::launch_autofocus(l, rc_dtype == BFPFFT_F16_BFP, rc, phi, static_cast<const float2*>(ha),
                                        a.tw, n_rg, static_cast<double*>(stats_out), grad_out, workspace,
                                        device_memory(rc), s);
  return cuda_status(e);
}

int sar_autofocus_entropy_arith(const void* rc, int rc_dtype, const float* phi, const void* ha, int64_t n_az,
                                int64_t n_rg, void* stats_out, void* workspace, size_t ws_bytes, int arith,
                                void* stream) {
  return autofocus_common(rc, rc_dtype, phi, ha, n_az, n_rg, nullptr, stats_out, workspace, ws_bytes, arith,
                          stream);
}

int sar_autofocus_grad_arith(const void* rc, int rc_dtype, const float* phi, const void* ha, int64_t n_az,
                             int64_t n_rg, float* grad_out, void* stats_out, void* workspace, size_t ws_bytes,
                             int arith, void* stream) {
  if (grad_out == nullptr) return BFPFFT_ERR_INVALID_ARG;
  return autofocus_common(rc, rc_dtype, phi, ha, n_az, n_rg, grad_out, stats_out, workspace, ws_bytes, arith,
                          stream);
}

int sar_autofocus_entropy(const void* rc, int rc_dtype, const float* phi, const void* ha, int64_t n_az,
                          int64_t n_rg, void* stats_out, void* workspace, size_t ws_bytes, void* stream) {
  return autofocus_common(rc, rc_dtype, phi, ha, n_az, n_rg, nullptr, stats_out, workspace, ws_bytes,
                          BFPFFT_ARITH_F32, stream);
}

int sar_autofocus_grad(const void* rc, int rc_dtype, const float* phi, const void* ha, int64_t n_az,
                       int64_t n_rg, float* grad_out, void* stats_out, void* workspace, size_t ws_bytes,
                       void* stream) {
  if (grad_out == nullptr) return BFPFFT_ERR_INVALID_ARG;
  return autofocus_common(rc, rc_dtype, phi, ha, n_az, n_rg, grad_out, stats_out, workspace, ws_bytes,
                          BFPFFT_ARITH_F32, stream);
}

size_t sar_point_target_workspace_bytes(int64_t n_az, int64_t n_rg) {
  if (n_az < 0 || n_rg < 0) return 0;
  return bfp::pt_workspace_bytes(n_az, n_rg);
}

int sar_point_target_metrics(const void* img, int img_dtype, int64_t n_az, int64_t n_rg, const int32_t* targets,
                             int64_t k, int guard, void* out, void* workspace, size_t ws_bytes, void* stream) {
  if (n_az < 64 || n_rg < 64 || k < 0 || k > 65535 || guard < 1) return BFPFFT_ERR_INVALID_ARG;
  if (img_dtype != BFPFFT_F32 && img_dtype != BFPFFT_F16_BFP && img_dtype != BFPFFT_F16_NAIVE)
    return BFPFFT_ERR_UNSUPPORTED;
  if (k == 0) return BFPFFT_OK;
  if (img == nullptr || targets == nullptr || out == nullptr || workspace == nullptr) return BFPFFT_ERR_INVALID_ARG;
  if (!aligned16(img) || !aligned16(out) || !aligned16(workspace)) return BFPFFT_ERR_MISALIGNED;
  if (ws_bytes < bfp::pt_workspace_bytes(n_az, n_rg)) return BFPFFT_ERR_INVALID_ARG;
  if (fault("launch")) return BFPFFT_ERR_CUDA;
  cudaError_t e = bfp::launch_point_target_metrics(img, img_dtype != BFPFFT_F32, n_az, n_rg, targets, int(k), guard,
                                                   static_cast<double*>(out), workspace,
                                                   static_cast<cudaStream_t>(stream));
  return cuda_status(e);
}

size_t bfp_sqnr_workspace_bytes(void) { return bfp::kMetricWorkspaceBytes; }

int bfp_sqnr_sums(const void* ref, int ref_dtype, const void* test, int test_dtype, int64_t count, void* sums_out,
                  void* workspace, size_t ws_bytes, void* stream) {
  if (count < 0) return BFPFFT_ERR_INVALID_ARG;
  if (ref_dtype != BFPFFT_F32 && ref_dtype != BFPFFT_F16_BFP && ref_dtype != BFPFFT_F16_NAIVE)
    return BFPFFT_ERR_UNSUPPORTED;
  if (test_dtype != BFPFFT_F32 && test_dtype != BFPFFT_F16_BFP && test_dtype != BFPFFT_F16_NAIVE)
    return BFPFFT_ERR_UNSUPPORTED;
  if (ref == nullptr || test == nullptr || sums_out == nullptr || workspace == nullptr)
    return BFPFFT_ERR_INVALID_ARG;
  if (!aligned16(ref) || !aligned16(test) || !aligned16(sums_out) || !aligned16(workspace))
    return BFPFFT_ERR_MISALIGNED;
  if (ws_bytes < size_t(bfp::metric_blocks(count)) * bfp::kMetricSums * sizeof(double))
    return BFPFFT_ERR_INVALID_ARG;
  if (fault("launch")) return BFPFFT_ERR_CUDA;
  cudaError_t e = bfp::launch_sqnr_sums(ref, ref_dtype != BFPFFT_F32, test, test_dtype != BFPFFT_F32, count,
                                        static_cast<double*>(workspace), static_cast<double*>(sums_out),
                                        static_cast<cudaStream_t>(stream));
  return cuda_status(e);
}

}  // extern "C"
