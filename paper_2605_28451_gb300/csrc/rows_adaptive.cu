// Row transforms with adaptive per-line block exponents (adaptive.cuh):
// plain forward / inverse on FP16 mantissas, and the forward-multiply-inverse
// spectral pipeline from complex64 values or FP16 mantissas.
#include "adaptive.cuh"
#include "launch.h"

namespace bfp {

cudaError_t launch_rows_adaptive_f16(int log2n, int mode, const RowArgs& a, cudaStream_t s) {
  switch (mode) {
    case kForward: return launch_rows_adaptive<__half2, kForward>(log2n, a, s);
    case kInverse: return launch_rows_adaptive<__half2, kInverse>(log2n, a, s);
    case kCompress: return launch_rows_adaptive<__half2, kCompress>(log2n, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_spectral_adaptive_c64(int log2n, const RowArgs& a, cudaStream_t s) {
  return launch_rows_adaptive<float2, kCompress>(log2n, a, s);
}

}  // namespace bfp
