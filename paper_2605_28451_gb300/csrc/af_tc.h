// Entropy autofocus on the tensor-core rows (af_tc.cu), 4096 pulses.
#pragma once

#include <cuda_runtime.h>

#include "fft_rows.cuh"

namespace bfp {

// Views into the caller's autofocus workspace (af_workspace_layout).
struct AfTcWorkspace {
  double* sq_part;   // [max_ctas][2]
  float* g_part;     // [max_ctas][4096]
  float* q_part;     // [max_ctas]
  float* qmax;       // [1]
  int max_ctas;
};

// Entropy statistics (stats[0..3] = S, sum q ln q, E, ln S) and, when grad is
// not null, dE/dphi[4096].  ph is the phase table e^{-j phi}; ra carries the
// status word, the pass-major twiddles of N = 4096 and the DFT-16 matrix.
cudaError_t launch_autofocus_tc(bool rc16, const void* rc, const float2* ph, const float2* ha, const RowArgs& ra,
                                long long n_rg, double* stats, float* grad, const AfTcWorkspace& ws, bool prefetch,
                                cudaStream_t s);

}  // namespace bfp
