// Range-Doppler imaging with RCMC and range-dependent azimuth filters (rda.cu).
#pragma once

#include <cuda_runtime.h>

namespace bfp {

struct RdaGeometry {
  double range_cell_m;     // slant-range sample spacing
  double prf_hz;           // pulse repetition frequency
  double wavelength_m;
  double speed_mps;        // platform speed
  double centre_range_m;   // slant range of range cell n_rg / 2
};

struct RdaArgs {
  const void* in;          // [lines][N] in the storage type
  void* out;               // [lines][N]; may equal in
  const float2* tw;        // pass-major FP32 twiddles of length N
  long long lines;
  long long other;         // the other dimension: n_az for RCMC lines, n_rg for azimuth lines
  RdaGeometry geo;
  int aperture;            // azimuth chirp length L (pulses)
  int range_dependent;     // azimuth lines: k_a(R) of the line's own range (else of the centre range)
  int peak_normalise;      // azimuth lines: H_r / max |H_r|
};

constexpr int kRdaMinLog2 = 8;
constexpr int kRdaMaxLog2 = 13;

// RCMC lines (along range, one per Doppler bin) and azimuth lines (along
// Doppler, one per range bin); f16 selects half2 storage, else float2.
cudaError_t launch_rcmc_rows(int log2n, bool f16, const RdaArgs& a, cudaStream_t s);
cudaError_t launch_azimuth_rows(int log2n, bool f16, const RdaArgs& a, cudaStream_t s);

}  // namespace bfp
