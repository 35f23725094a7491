// SAR compression, row-major in, corner-turned out (range compression into
// [n_rg][n_az], or azimuth compression of a transposed intermediate).
#include "sar_dispatch.cuh"

namespace bfp {

cudaError_t launch_sar_nt(int log2n, bool in16, bool out16, bool naive, const RowArgs& a, cudaStream_t s) {
  return sar_variant<false, true>(log2n, in16, out16, naive, a, s);
}

}  // namespace bfp
