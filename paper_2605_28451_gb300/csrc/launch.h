// Host-side launch entry points of the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include "fft_rows.cuh"

namespace bfp {

// float2 -> float2 rows: mode in {kForward, kInverse, kCompress}.
cudaError_t launch_rows_f32(int log2n, int mode, const RowArgs& a, cudaStream_t s);
// __half2 -> __half2 rows; naive selects the unshifted inverse (Section III-B).
cudaError_t launch_rows_f16(int log2n, int mode, bool naive, const RowArgs& a, cudaStream_t s);
// Mixed-storage compress: float2 raw -> __half2 out, or __half2 raw -> float2 out.
cudaError_t launch_compress_c64_to_f16(int log2n, bool naive, const RowArgs& a, cudaStream_t s);
cudaError_t launch_compress_f16_to_c64(int log2n, const RowArgs& a, cudaStream_t s);
// FP8 rows (fmt 0 = E4M3, 1 = E5M2); mode in {kForward, kInverse}.
cudaError_t launch_rows_fp8(int log2n, int mode, int fmt, const RowArgs& a, cudaStream_t s);

// Adaptive per-line block exponents (adaptive.cuh), log2n in [4, 14]: FP16
// mantissas with a.in_exp (may be null) in, FP16 mantissas and a.out_exp out;
// mode in {kForward, kInverse, kCompress}.  The c64 form reads complex64
// values and runs the compress (spectral) mode.
constexpr int kAdaptiveMaxLog2 = 14;
cudaError_t launch_rows_adaptive_f16(int log2n, int mode, const RowArgs& a, cudaStream_t s);
cudaError_t launch_spectral_adaptive_c64(int log2n, const RowArgs& a, cudaStream_t s);

// Rows in 16-bit arithmetic (fft_half.cuh), log2n in [4, 14]; a.tw16 holds the
// table written by launch_twiddles16 (n entries of 8 bytes).
constexpr int kRows16MaxLog2 = 14;
cudaError_t launch_rows16_f16(int log2n, int mode, bool naive, const RowArgs& a, cudaStream_t s);
cudaError_t launch_rows16_bf16(int log2n, int mode, const RowArgs& a, cudaStream_t s);
// SAR compression lines in FP16 arithmetic (log2n in [8, 14]): in32 reads a
// complex64 input; naive drops the 1/N shift (Section III-B).
cudaError_t launch_rows16_compress_f16(int log2n, bool in32, bool naive, const RowArgs& a, cudaStream_t s);
cudaError_t launch_twiddles16(void* tw, int n, bool bf16);
// SAR compression lines of 4096 points on the tensor cores (tc_fft.cuh): FP16
// operands, FP32 accumulation; in32 reads a complex64 input; FP16 output rows.
// a.tc_b holds the DFT-16 matrix, a.h the filter spectrum.
cudaError_t launch_tc_compress(bool in32, const RowArgs& a, cudaStream_t s);
// Dense FP8 rows of 4096 points on the tensor cores (fmt 0: E4M3, 1: E5M2),
// with the block exponents in a.in_scale / a.out_scale.
cudaError_t launch_tc_fp8(int mode, int fmt, const RowArgs& a, cudaStream_t s);

// SAR compression lines (Section VI, Fig. 1): float2 or __half2 in and out,
// optional naive FP16 output, optional cluster corner turn on load / store.
// Supported log2n: [kSarMinLog2, 14].
constexpr int kSarMinLog2 = 8;
cudaError_t launch_sar(int log2n, bool in16, bool out16, bool naive, bool tload, bool tstore,
                       const RowArgs& a, cudaStream_t s);
cudaError_t launch_sar_nn(int log2n, bool in16, bool out16, bool naive, const RowArgs& a, cudaStream_t s);
cudaError_t launch_sar_nt(int log2n, bool in16, bool out16, bool naive, const RowArgs& a, cudaStream_t s);
cudaError_t launch_sar_tt(int log2n, bool in16, bool out16, bool naive, const RowArgs& a, cudaStream_t s);

// out[c][r] = in[r][c] for a row-major [rows][cols] array of 4- or 8-byte
// elements (half2 / float2).
cudaError_t launch_transpose(const void* in, void* out, long long rows, long long cols, int elem_bytes,
                             cudaStream_t s);


}  // namespace bfp
