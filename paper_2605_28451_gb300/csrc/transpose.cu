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
//
// Each CTA takes tiles b, b + gridDim.x, ... and loads its next tile into
// registers before it writes the current one out, so the loads of one tile
// overlap the shared-memory reads and global stores of the one before.
template <class T>
struct TileIo {
  static constexpr int VEC = 16 / sizeof(T);
  static constexpr int TILE = 16 * VEC;
  static constexpr int ROUNDS = TILE / 16;
  long long rows, cols, col_tiles;

  __device__ void origin(long long b, long long& r0, long long& c0) const {
    c0 = (b % col_tiles) * TILE;
    r0 = (b / col_tiles) * TILE;
  }
  // This thread's share of tile b: ROUNDS rows of VEC consecutive elements.
  __device__ void load(const T* __restrict__ in, long long b, int lr, int rr, T (&e)[ROUNDS][VEC]) const {
    long long r0, c0;
    origin(b, r0, c0);
    const bool vec = r0 + TILE <= rows && c0 + TILE <= cols && cols % VEC == 0;
#pragma unroll
    for (int k = 0; k < ROUNDS; ++k) {
      const long long r = r0 + rr + 16 * k, c = c0 + lr * VEC;
      if (vec) {
        *reinterpret_cast<uint4*>(e[k]) = __ldcs(reinterpret_cast<const uint4*>(in + r * cols + c));
      } else {
#pragma unroll
        for (int i = 0; i < VEC; ++i) {
          if (r < rows && c + i < cols) e[k][i] = in[r * cols + c + i];
        }
      }
    }
  }
};

template <class T>
__global__ void __launch_bounds__(256, 8) transpose_kernel(const T* __restrict__ in, T* __restrict__ out,
                                                        long long rows, long long cols, long long col_tiles,
                                                        long long tiles) {
  using Io = TileIo<T>;
  constexpr int VEC = Io::VEC, TILE = Io::TILE, ROUNDS = Io::ROUNDS;
  __shared__ T tile[TILE][TILE + 1];
  const Io io{rows, cols, col_tiles};
  const int lr = threadIdx.x % 16, rr = threadIdx.x / 16;
  long long b = blockIdx.x;
  if (b >= tiles) return;
  T e[ROUNDS][VEC];
  io.load(in, b, lr, rr, e);
  for (; b < tiles; b += gridDim.x) {
#pragma unroll
    for (int k = 0; k < ROUNDS; ++k) {
#pragma unroll
      for (int i = 0; i < VEC; ++i) tile[rr + 16 * k][lr * VEC + i] = e[k][i];
    }
    __syncthreads();
    const long long nb = b + gridDim.x;
    if (nb < tiles) io.load(in, nb, lr, rr, e);        // in flight while this tile is written
    long long r0, c0;
    io.origin(b, r0, c0);
    const bool vec_out = r0 + TILE <= rows && c0 + TILE <= cols && rows % VEC == 0;
#pragma unroll
    for (int k = 0; k < ROUNDS; ++k) {
      const int tc = rr + 16 * k;                      // column of the tile = row of the output
      const long long oc = c0 + tc, orow = r0 + lr * VEC;
      T w[VEC];
#pragma unroll
      for (int i = 0; i < VEC; ++i) w[i] = tile[lr * VEC + i][tc];
      if (vec_out) {
        __stcs(reinterpret_cast<uint4*>(out + oc * rows + orow), *reinterpret_cast<const uint4*>(w));
      } else {
#pragma unroll
        for (int i = 0; i < VEC; ++i) {
          if (oc < cols && orow + i < rows) out[oc * rows + orow + i] = w[i];
        }
      }
    }
    __syncthreads();                                   // the tile buffer is free for the next tile
  }
}

}  // namespace

cudaError_t launch_transpose(const void* in, void* out, long long rows, long long cols, int elem_bytes,
                             cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  if (elem_bytes != 4 && elem_bytes != 8) return cudaErrorInvalidValue;
  const int tile = elem_bytes == 4 ? 64 : 32;
  const long long gx = (cols + tile - 1) / tile, gy = (rows + tile - 1) / tile;
  const long long tiles = gx * gy;
  // Resident CTAs of the kernel on this device, once per element size.
  static int resident[2] = {0, 0};
  int& res = resident[elem_bytes == 4 ? 0 : 1];
  if (res == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = elem_bytes == 4
              ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, transpose_kernel<unsigned int>, 256, 0)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, transpose_kernel<float2>, 256, 0);
    if (e != cudaSuccess) return e;
    res = sms * per_sm > 0 ? sms * per_sm : 1;
  }
  // Every CTA takes the same number of tiles (the last ones one fewer at most).
  const long long per_cta = (tiles + res - 1) / res;
  const long long grid = (tiles + per_cta - 1) / per_cta;
  const dim3 block{256u, 1u, 1u};
  if (elem_bytes == 4) {
    transpose_kernel<unsigned int><<<unsigned(grid), block, 0, s>>>(
        static_cast<const unsigned int*>(in), static_cast<unsigned int*>(out), rows, cols, gx, tiles);
  } else {
    transpose_kernel<float2><<<unsigned(grid), block, 0, s>>>(static_cast<const float2*>(in),
                                                             static_cast<float2*>(out), rows, cols, gx, tiles);
  }
  return cudaGetLastError();
}

}  // namespace bfp
