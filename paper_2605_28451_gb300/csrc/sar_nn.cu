// SAR compression, row-major in and out (range compression, no corner turn).
#include "sar_dispatch.cuh"

namespace bfp {

cudaError_t launch_sar_nn(int log2n, bool in16, bool out16, bool naive, const RowArgs& a, cudaStream_t s) {
  return sar_variant<false, false>(log2n, in16, out16, naive, a, s);
}

cudaError_t launch_sar(int log2n, bool in16, bool out16, bool naive, bool tload, bool tstore,
                       const RowArgs& a, cudaStream_t s) {
  if (log2n < kSarMinLog2 || log2n > 14) return cudaErrorInvalidValue;
  if (!tload && !tstore) return launch_sar_nn(log2n, in16, out16, naive, a, s);
  if (!tload && tstore) return launch_sar_nt(log2n, in16, out16, naive, a, s);
  if (tload && tstore) return launch_sar_tt(log2n, in16, out16, naive, a, s);
  return cudaErrorInvalidValue;
}

}  // namespace bfp
