// bfp_sqnr_sums_noalloc: the FP64 SQNR reduction of bfp_sqnr_sums with its
// scratch in a fixed device array inside this library, for callers that
// cannot allocate device memory or hand the library a workspace.
//
// Scratch: g_sqnr_scratch, kNoAllocBlocks x 5 FP64 partial sums (160 KB),
// defined at file scope, so every GPU that loads the library holds it until
// the process exits.  Stage 1 gives each block kNoAllocPointsPerBlock points
// and writes one partial per block; stage 2 adds them.  A call therefore
// takes at most kNoAllocBlocks * kNoAllocPointsPerBlock = 16,777,216 points
// (a 4096 x 4096 image); larger counts are rejected.
//
// Host code never uses g_sqnr_scratch's name as an address: that name is a
// host-side stand-in.  The device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) on the first call made on
// that device, checked, cached, and passed to the kernels.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "bfpfft.h"
#include "metrics.h"

namespace {

constexpr int kNoAllocBlocks = 4096;
constexpr long long kNoAllocPointsPerBlock = 4096;     // 256 threads x 16 points
constexpr long long kNoAllocMaxPoints = kNoAllocBlocks * kNoAllocPointsPerBlock;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_sqnr_scratch[kNoAllocBlocks * bfp::kMetricSums];

std::mutex g_scratch_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return BFPFFT_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return BFPFFT_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sqnr_scratch) != cudaSuccess || p == nullptr) return BFPFFT_ERR_CUDA;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return BFPFFT_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" {

long long bfp_sqnr_sums_noalloc_max_count(void) { return kNoAllocMaxPoints; }

int bfp_sqnr_sums_noalloc(const void* ref, int ref_dtype, const void* test, int test_dtype, int64_t count,
                          void* sums_out, void* stream) {
  if (count < 0) return BFPFFT_ERR_INVALID_ARG;
  if (count > kNoAllocMaxPoints) return BFPFFT_ERR_UNSUPPORTED;
  if (ref_dtype != BFPFFT_F32 && ref_dtype != BFPFFT_F16_BFP && ref_dtype != BFPFFT_F16_NAIVE)
    return BFPFFT_ERR_UNSUPPORTED;
  if (test_dtype != BFPFFT_F32 && test_dtype != BFPFFT_F16_BFP && test_dtype != BFPFFT_F16_NAIVE)
    return BFPFFT_ERR_UNSUPPORTED;
  if (ref == nullptr || test == nullptr || sums_out == nullptr) return BFPFFT_ERR_INVALID_ARG;
  if (!aligned16(ref) || !aligned16(test) || !aligned16(sums_out)) return BFPFFT_ERR_MISALIGNED;
  double* scratch = nullptr;
  int st = scratch_for_current_device(&scratch);
  if (st != BFPFFT_OK) return st;
  long long blocks = (count + kNoAllocPointsPerBlock - 1) / kNoAllocPointsPerBlock;
  if (blocks < 1) blocks = 1;
  // Stage 1 writes every partial that stage 2 reads, so nothing left over
  // from an earlier call needs clearing.
  cudaError_t e = bfp::launch_sqnr_sums_blocks(ref, ref_dtype != BFPFFT_F32, test, test_dtype != BFPFFT_F32,
                                               count, scratch, int(blocks), static_cast<double*>(sums_out),
                                               static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? BFPFFT_OK : BFPFFT_ERR_CUDA;
}

}  // extern "C"
