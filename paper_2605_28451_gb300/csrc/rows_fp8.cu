// FP8-storage row transforms (Section VII): E4M3 / E5M2 in HBM, FP32 compute,
// static power-of-two block exponents applied at load and store.
#include "launch.h"

namespace bfp {

cudaError_t launch_rows_fp8(int log2n, int mode, int fmt, const RowArgs& a, cudaStream_t s) {
  using A = Fp8x2<E4M3>;
  using B = Fp8x2<E5M2>;
  if (fmt == 0) {
    if (mode == kForward) return launch_rows<A, A, kForward, false, true>(log2n, a, s);
    if (mode == kInverse) return launch_rows<A, A, kInverse, false, true>(log2n, a, s);
  } else if (fmt == 1) {
    if (mode == kForward) return launch_rows<B, B, kForward, false, true>(log2n, a, s);
    if (mode == kInverse) return launch_rows<B, B, kInverse, false, true>(log2n, a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace bfp
