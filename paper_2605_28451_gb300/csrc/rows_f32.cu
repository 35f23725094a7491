// FP32-storage row transforms (the comparison path of Section V, Table II).
#include "launch.h"

namespace bfp {

cudaError_t launch_rows_f32(int log2n, int mode, const RowArgs& a, cudaStream_t s) {
  switch (mode) {
    case kForward: return launch_rows<float2, float2, kForward, false, false>(log2n, a, s);
    case kInverse: return launch_rows<float2, float2, kInverse, false, false>(log2n, a, s);
    case kCompress: return launch_rows<float2, float2, kCompress, false, false>(log2n, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_compress_f16_to_c64(int log2n, const RowArgs& a, cudaStream_t s) {
  return launch_rows<__half2, float2, kCompress, false, false>(log2n, a, s);
}

}  // namespace bfp
