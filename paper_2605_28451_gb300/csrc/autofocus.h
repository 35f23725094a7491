// Entropy autofocus launchers.
#pragma once

#include <cuda_runtime.h>

namespace bfp {

constexpr int kAfMaxCtas = 640;   // cap on persistent CTAs (sizes the partial-gradient workspace)
constexpr int kAfMinLog2 = 8;
constexpr int kAfMaxLog2 = 13;

// Workspace bytes for azimuth length n_az (any number of range bins).
size_t af_workspace_bytes(long long n_az);

// Entropy statistics (stats[0..3] = S, sum q ln q, E, ln S; device) and, when
// grad != nullptr, dE/dphi (grad[n_az], device).  rc is [n_rg][2^log2n].
cudaError_t launch_autofocus(int log2n, bool rc16, const void* rc, const float* phi, const float2* ha,
                             const float2* tw, long long n_rg, double* stats, float* grad, void* workspace,
                             bool prefetch, cudaStream_t s);

}  // namespace bfp
