// FP16-storage row transforms: the block-floating-point path (Eq. 1) and the
// naive unshifted path of Section III-B.
#include "launch.h"
#include "tc_fft.cuh"

namespace bfp {

cudaError_t launch_rows_f16(int log2n, int mode, bool naive, const RowArgs& a, cudaStream_t s) {
  if (naive) {
    switch (mode) {
      case kForward: return launch_rows<__half2, __half2, kForward, false, false>(log2n, a, s);
      case kInverse: return launch_rows<__half2, __half2, kInverse, true, false>(log2n, a, s);
      case kCompress: return launch_rows<__half2, __half2, kCompress, true, false>(log2n, a, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (mode) {
    case kForward: return launch_rows<__half2, __half2, kForward, false, false>(log2n, a, s);
    case kInverse: return launch_rows<__half2, __half2, kInverse, false, false>(log2n, a, s);
    case kCompress: return launch_rows<__half2, __half2, kCompress, false, false>(log2n, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_compress_c64_to_f16(int log2n, bool naive, const RowArgs& a, cudaStream_t s) {
  if (naive) return launch_rows<float2, __half2, kCompress, true, false>(log2n, a, s);
  return launch_rows<float2, __half2, kCompress, false, false>(log2n, a, s);
}

cudaError_t launch_tc_compress(bool in32, const RowArgs& a, cudaStream_t s) {
  if (a.tc_b == nullptr || a.h == nullptr) return cudaErrorInvalidValue;
  return in32 ? launch_tc_kernel<kCompress, float2>(a, s) : launch_tc_kernel<kCompress, __half2>(a, s);
}

}  // namespace bfp
