// Out-of-place transpose of a row-major [rows][cols] array of complex values
// (4-byte half2 or 8-byte float2): out[c][r] = in[r][c].
//
// The SAR pipeline (Fig. 1) compresses range lines (rows of the raw data) and
// azimuth lines (columns); between the two the data is turned.  One CTA moves
// a tile through padded shared memory; both the reads (tile rows) and the
// writes (rows of the turned tile) are 16-byte vectors, 256 contiguous bytes
// per half warp.
#include <cuda_runtime.h>

#include <cstdint>

#include "launch.h"

namespace bfp {

namespace {

// Tiles of TILE x TILE elements, TILE * sizeof(T) = 256 bytes: 64 x 64 half2
// or 32 x 32 float2.  256 threads: 16 per tile row (one 16-byte vector each),
// 16 rows per round.  Vector accesses need the row pitch to be a multiple of
// 16 bytes; ragged edge tiles and other pitches use element accesses.
template <class T>
__global__ void __launch_bounds__(256) transpose_kernel(const T* __restrict__ in, T* __restrict__ out,
                                                        long long rows, long long cols, long long col_tiles) {
  constexpr int VEC = 16 / sizeof(T);
  constexpr int TILE = 16 * VEC;
  __shared__ T tile[TILE][TILE + 1];
  using V = uint4;
  const long long b = blockIdx.x;                  // one-dimensional grid, column tiles fastest
  const long long c0 = (b % col_tiles) * TILE, r0 = (b / col_tiles) * TILE;
  const int lr = threadIdx.x % 16, rr = threadIdx.x / 16;
  const bool full = r0 + TILE <= rows && c0 + TILE <= cols;
  const bool vec_in = full && cols % VEC == 0, vec_out = full && rows % VEC == 0;
#pragma unroll
  for (int k = 0; k < TILE / 16; ++k) {
    const int tr = rr + 16 * k;
    const long long r = r0 + tr, c = c0 + lr * VEC;
    T e[VEC];
    if (vec_in) {
      const V q = __ldcs(reinterpret_cast<const V*>(in + r * cols + c));
      *reinterpret_cast<V*>(e) = q;
    } else {
#pragma unroll
      for (int i = 0; i < VEC; ++i) {
        if (r < rows && c + i < cols) e[i] = in[r * cols + c + i];
      }
    }
#pragma unroll
    for (int i = 0; i < VEC; ++i) tile[tr][lr * VEC + i] = e[i];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < TILE / 16; ++k) {
    const int tc = rr + 16 * k;                      // column of the tile = row of the output
    const long long oc = c0 + tc, orow = r0 + lr * VEC;
    T e[VEC];
#pragma unroll
    for (int i = 0; i < VEC; ++i) e[i] = tile[lr * VEC + i][tc];
    if (vec_out) {
      __stcs(reinterpret_cast<V*>(out + oc * rows + orow), *reinterpret_cast<const V*>(e));
    } else {
#pragma unroll
      for (int i = 0; i < VEC; ++i) {
        if (oc < cols && orow + i < rows) out[oc * rows + orow + i] = e[i];
      }
    }
  }
}

}  // namespace

cudaError_t launch_transpose(const void* in, void* out, long long rows, long long cols, int elem_bytes,
                             cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const int tile = elem_bytes == 4 ? 64 : 32;
  const long long gx = (cols + tile - 1) / tile, gy = (rows + tile - 1) / tile;
  if (gx * gy > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const dim3 grid{unsigned(gx * gy), 1u, 1u}, block{256u, 1u, 1u};
  if (elem_bytes == 4) {
    transpose_kernel<unsigned int><<<grid, block, 0, s>>>(static_cast<const unsigned int*>(in),
                                                          static_cast<unsigned int*>(out), rows, cols, gx);
  } else if (elem_bytes == 8) {
    transpose_kernel<float2>
        <<<grid, block, 0, s>>>(static_cast<const float2*>(in), static_cast<float2*>(out), rows, cols, gx);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace bfp
