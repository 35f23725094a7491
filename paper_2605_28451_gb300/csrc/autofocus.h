// Entropy autofocus launchers.
#pragma once

#include <cuda_runtime.h>

namespace bfp {

constexpr int kAfMaxCtas = 1216;  // cap on persistent CTAs (sizes the partial-gradient workspace)
constexpr int kAfMinLog2 = 8;
constexpr int kAfMaxLog2 = 13;

// Workspace bytes for azimuth length n_az (any number of range bins).
size_t af_workspace_bytes(long long n_az);

// The workspace's parts: per-CTA FP64 entropy partials [kAfMaxCtas][2],
// per-CTA pulse gradients [kAfMaxCtas][n_az], the phase table [n_az], the
// per-CTA largest q [kAfMaxCtas] and their maximum [1].
struct AfWorkspaceLayout {
  double* sq_part;
  float* g_part;
  float2* ph;
  float* q_part;
  float* qmax;
};
AfWorkspaceLayout af_workspace_layout(void* workspace, long long n_az);

// Pieces shared with the tensor-core autofocus: the phase table e^{-j phi},
// the entropy statistics from per-CTA partials, and the sum of per-CTA pulse
// gradients.
cudaError_t af_phase_table(const float* phi, float2* ph, long long n_az, cudaStream_t s);
cudaError_t af_entropy_stats(const double* sq_part, int grid, double* stats, cudaStream_t s);
cudaError_t af_gradient_sum(const float* g_part, int grid, int n_az, float* grad, cudaStream_t s);

// Entropy statistics (stats[0..3] = S, sum q ln q, E, ln S; device) and, when
// grad != nullptr, dE/dphi (grad[n_az], device).  rc is [n_rg][2^log2n].
cudaError_t launch_autofocus(int log2n, bool rc16, const void* rc, const float* phi, const float2* ha,
                             const float2* tw, long long n_rg, double* stats, float* grad, void* workspace,
                             bool prefetch, cudaStream_t s);

}  // namespace bfp
