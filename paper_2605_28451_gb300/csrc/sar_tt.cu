// SAR compression along columns of a row-major matrix: corner turn on load and
// on store (azimuth compression of [n_az][n_rg] data in place of layout).
#include "sar_dispatch.cuh"

namespace bfp {

cudaError_t launch_sar_tt(int log2n, bool in16, bool out16, bool naive, const RowArgs& a, cudaStream_t s) {
  return sar_variant<true, true>(log2n, in16, out16, naive, a, s);
}

}  // namespace bfp
