// FP8-storage rows on the tensor cores, N = 4096: E4M3 / E5M2 pairs in HBM,
// converted exactly to FP16 operands, FP32 accumulation (Section VI's FP16
// multiply / FP32 accumulate with Section VII's FP8 storage), the static
// block exponents of the FP8 plans applied in FP32 after the first pass.
#include "launch.h"
#include "tc_fft.cuh"

namespace bfp {

cudaError_t launch_tc_fp8(int mode, int fmt, const RowArgs& a, cudaStream_t s) {
  using A = Fp8x2<E4M3>;
  using B = Fp8x2<E5M2>;
  if (a.tc_b == nullptr || a.in_stride != 4096 || a.out_stride != 4096) return cudaErrorInvalidValue;
  if (fmt == 0) {
    if (mode == kForward) return launch_tc_kernel<kForward, A, A>(a, s);
    if (mode == kInverse) return launch_tc_kernel<kInverse, A, A>(a, s);
  } else if (fmt == 1) {
    if (mode == kForward) return launch_tc_kernel<kForward, B, B>(a, s);
    if (mode == kInverse) return launch_tc_kernel<kInverse, B, B>(a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace bfp
