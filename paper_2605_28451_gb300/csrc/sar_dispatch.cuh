// Shared dispatch for the SAR compression kernels of one layout variant.
#pragma once

#include "launch.h"

namespace bfp {

template <class TIn, class TOut, bool NAIVE, bool TLOAD, bool TSTORE>
cudaError_t sar_sized(int log2n, const RowArgs& a, cudaStream_t s) {
  switch (log2n) {
    case 8: return launch_rows_n<256, TIn, TOut, kCompress, NAIVE, false, TLOAD, TSTORE>(a, s);
    case 9: return launch_rows_n<512, TIn, TOut, kCompress, NAIVE, false, TLOAD, TSTORE>(a, s);
    case 10: return launch_rows_n<1024, TIn, TOut, kCompress, NAIVE, false, TLOAD, TSTORE>(a, s);
    case 11: return launch_rows_n<2048, TIn, TOut, kCompress, NAIVE, false, TLOAD, TSTORE>(a, s);
    case 12: return launch_rows_n<4096, TIn, TOut, kCompress, NAIVE, false, TLOAD, TSTORE>(a, s);
    case 13: return launch_rows_n<8192, TIn, TOut, kCompress, NAIVE, false, TLOAD, TSTORE>(a, s);
    case 14: return launch_rows_n<16384, TIn, TOut, kCompress, NAIVE, false, TLOAD, TSTORE>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <bool TLOAD, bool TSTORE>
cudaError_t sar_variant(int log2n, bool in16, bool out16, bool naive, const RowArgs& a, cudaStream_t s) {
  if (!out16 && naive) return cudaErrorInvalidValue;
  if (in16) {
    if (!out16) return sar_sized<__half2, float2, false, TLOAD, TSTORE>(log2n, a, s);
    if (naive) return sar_sized<__half2, __half2, true, TLOAD, TSTORE>(log2n, a, s);
    return sar_sized<__half2, __half2, false, TLOAD, TSTORE>(log2n, a, s);
  }
  if (!out16) return sar_sized<float2, float2, false, TLOAD, TSTORE>(log2n, a, s);
  if (naive) return sar_sized<float2, __half2, true, TLOAD, TSTORE>(log2n, a, s);
  return sar_sized<float2, __half2, false, TLOAD, TSTORE>(log2n, a, s);
}

}  // namespace bfp
