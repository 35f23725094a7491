// Long lines as two streaming passes (twopass.cu).
#pragma once

#include <cuda_runtime.h>

namespace bfp {

struct TwoPassArgs {
  const void* in;
  void* out;
  void* scratch;              // intermediate of chunk_lines lines (twopass_scratch_bytes)
  const long long* line_off;  // point offset of every line, or nullptr for dense lines (line l at l N)
  long long first_line;       // first line handled by this launch pair (set per chunk)
  long long count;            // lines handled by this launch pair (set per chunk)
  long long lines;            // lines of the call
  long long chunk_lines;      // lines per launch pair (<= 0: all at once)
  const float2* tw_col;       // pass-major FP32 twiddles of length N1 (the column DFT)
  const float2* tw_row;       // pass-major FP32 twiddles of length 256 (the row DFT)
  const float2* tw_4step;     // W_N^{n2 k1} at k1 * 256 + n2, k1 < N1, n2 < 256
  float in_scale;             // FP8 block exponents (as RowArgs)
  float out_scale;
  int* finite_flag;           // BFPFFT_CHECK_FINITE
  int pf_ahead;               // > 0: each CTA prefetches into L2 what the CTA pf_ahead blocks later reads
};

// Storage kinds as the uneven kernel: 0 FP32, 1 FP16, 2 E4M3, 3 E5M2.
// log2n: 15 or 16; mode: kForward or kInverse.
cudaError_t launch_twopass(int kind, int log2n, int mode, const TwoPassArgs& a, cudaStream_t s);
size_t twopass_scratch_bytes(int kind, long long lines_per_chunk, int log2n);

}  // namespace bfp
