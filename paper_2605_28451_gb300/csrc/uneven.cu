// Uneven batches: many transforms of different power-of-two lengths (16 ..
// 65536) in ONE persistent launch.
//
// Work is cut into tasks of 65,536 points of one length: a task is one line
// of 65536, four of 16384, ..., sixteen of 4096, ..., 4096 of 16.  The grid is
// made of thread-block clusters of 16 CTAs x 256 threads (16 points per
// thread, the register layout of fft_rows.cuh).  Cluster k takes tasks k,
// k + clusters, ... (all tasks are the same size); no CTA ever waits for
// another cluster.  Within a task:
//   N <= 4096   every CTA transforms 4096 / N lines in its own shared memory;
//   N >= 8192   a line spans N / 4096 CTAs of the cluster: the four-step line
//               of fft_rows.cuh (one exchange through distributed shared
//               memory, then local 4096-point transforms).
// Tasks are ordered largest length first so the short tasks fill the tail.
// Storage: FP16 (BFP shift before the inverse), FP32, or FP8 with the static
// block exponents of the uniform plans; arithmetic FP32.
#include <cooperative_groups.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "fft_rows.cuh"
#include "uneven.h"

namespace bfp {

namespace {

constexpr int kCta = 256;
constexpr int kClusterCtas = 16;
constexpr int kSlab = 4096;     // points of one line per CTA (N >= 4096)

// Returns false when a bounded wait of a four-step line expired (the CTA
// then stops working, see uneven_kernel); `pending` as in fourstep_line.
template <class TS, int MODE, bool SCALED, bool H16ROW, int LOG2N>
__device__ __noinline__ bool run_task(const UnevenArgs& a, const UnevenTask& tk, int rank, float2* smem,
                                      uint64_t* bar, uint32_t& phase, int& pending) {
  constexpr int N = 1 << LOG2N;
  constexpr int P = kPointsPerThread, T = N / P;
  RowArgs ra{};
  ra.tw = a.tw[LOG2N];
  ra.status = a.status;
  ra.finite_flag = a.finite_flag;
  const int s = (LOG2N + 1) / 2;                        // FP8 block exponent
  ra.in_scale = SCALED && MODE == kInverse ? float(1 << s) : 1.f;
  ra.out_scale = SCALED && MODE == kForward ? 1.f / float(1 << s) : 1.f;
  float2 v[P];
  if constexpr (N <= kSlab) {
    constexpr int G = kCta / T;                          // lines per CTA
    const int g = threadIdx.x / T;
    const int t = threadIdx.x - g * T;
    const int idx = rank * G + g;                        // line within the task
    const bool active = idx < tk.count;
    const long long off = active ? a.line_off[tk.first + idx] : 0;
    if (active) {
      const TS* in = static_cast<const TS*>(a.in) + off + t;
#pragma unroll
      for (int m = 0; m < P; ++m) v[m] = Storage<TS>::load(in + T * m);
    } else {
#pragma unroll
      for (int m = 0; m < P; ++m) v[m] = make_float2(0.f, 0.f);
    }
    row_compute_x<N, MODE, false, SCALED>(v, ra, LocalXch{smem + g * pad16(N)}, t);
    if (active) {
      TS* out = static_cast<TS*>(a.out) + off + t;
#pragma unroll
      for (int m = 0; m < P; ++m) Storage<TS>::store(out + T * m, v[m]);
      check_finite<Storage<TS>, P>(a.finite_flag, [&](int m) { return v[m]; });
    }
    return true;
  } else {
    constexpr int C = N / kSlab;                         // CTAs per line
    const int idx = rank / C;                            // line within the task
    const int base = idx * C;
    const bool active = idx < tk.count;
    const long long off = active ? a.line_off[tk.first + idx] : 0;
    ra.tw_line = a.tw[12];
    ra.tw_4step = a.tw4[LOG2N];
    return fourstep_line<C, TS, MODE, SCALED, H16ROW>(ra, static_cast<const TS*>(a.in) + off,
                                              static_cast<TS*>(a.out) + off, smem, bar, bar + 1, phase, pending,
                                              rank - base, base, active);
  }
}

// Prefetch into L2 the lines this CTA transforms in `task` (the cluster's next
// task, about one resident wave ahead): for N <= 4096 the first thread of each
// line group prefetches its line, for longer lines thread 0 its 4096-point
// share.  Line offsets and lengths are multiples of 16 points, so every
// prefetch is 16-byte aligned and sized.
template <class TS>
__device__ __forceinline__ void prefetch_task(const UnevenArgs& a, int task, int rank) {
  if (task >= a.num_tasks) return;
  const UnevenTask tk = a.tasks[task];
  const int n = 1 << tk.log2n;
  const TS* in = static_cast<const TS*>(a.in);
  if (n <= kSlab) {
    const int T = n / kPointsPerThread, G = kCta / T;
    const int g = threadIdx.x / T, t = threadIdx.x - g * T;
    const int idx = rank * G + g;
    if (t == 0 && idx < tk.count) prefetch_l2_bulk(in + a.line_off[tk.first + idx], uint32_t(n * sizeof(TS)));
  } else {
    const int C = n / kSlab;
    const int idx = rank / C, c = rank - idx * C;
    if (threadIdx.x == 0 && idx < tk.count)
      prefetch_l2_bulk(in + a.line_off[tk.first + idx] + c * kSlab, uint32_t(kSlab * sizeof(TS)));
  }
}

// H16ROW (FP16 storage only): four-step lines exchange their rows as FP16
// words.
template <class TS, int MODE, bool SCALED, bool H16ROW>
// Four CTAs per SM (64 registers) where their shared memory fits (FP16
// storage), else three.
__global__ void __launch_bounds__(kCta, uneven_smem_bytes<TS>() * 4 <= 220 * 1024 ? 4 : 3)
    uneven_kernel(const UnevenArgs a) {
  extern __shared__ float2 smem_u[];
  __shared__ __align__(8) uint64_t bar[2];   // row and output exchanges of four-step lines
  auto cluster = cooperative_groups::this_cluster();
  const int rank = int(cluster.block_rank());
  const int cluster_id = int(blockIdx.x) / kClusterCtas;
  const int clusters = int(gridDim.x) / kClusterCtas;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // Peers running, mbarriers initialised (published by their release fence).
  cluster_arrive_relaxed();
  cluster_wait_acquire();
  uint32_t phase = 0;
  // A bounded wait that expired (recorded in a.status) puts this CTA in abort
  // mode: it stops loading, sending and waiting, but walks the rest of the
  // task list so that it passes exactly the cluster barriers its peers pass
  // (the barrier decisions below depend on the task list only).  A peer that
  // waits for data this CTA no longer sends expires once (one bound) and
  // aborts too, so a failing launch ends after a few bounds instead of one
  // bound per remaining task.
  bool aborted = false;
  int pending = 0;
  // Tasks hold 65,536 points each, so a static round-robin over the clusters
  // balances the work; no counter or broadcast is needed.
  if (a.prefetch) prefetch_task<TS>(a, cluster_id, rank);
  for (int task = cluster_id; task < a.num_tasks; task += clusters) {
    const UnevenTask tk = a.tasks[task];
    if (!aborted) {
      if (a.prefetch) prefetch_task<TS>(a, task + clusters, rank);
      bool ok = true;
      switch (tk.log2n) {
        case 4: ok = run_task<TS, MODE, SCALED, H16ROW, 4>(a, tk, rank, smem_u, bar, phase, pending); break;
        case 5: ok = run_task<TS, MODE, SCALED, H16ROW, 5>(a, tk, rank, smem_u, bar, phase, pending); break;
        case 6: ok = run_task<TS, MODE, SCALED, H16ROW, 6>(a, tk, rank, smem_u, bar, phase, pending); break;
        case 7: ok = run_task<TS, MODE, SCALED, H16ROW, 7>(a, tk, rank, smem_u, bar, phase, pending); break;
        case 8: ok = run_task<TS, MODE, SCALED, H16ROW, 8>(a, tk, rank, smem_u, bar, phase, pending); break;
        case 9: ok = run_task<TS, MODE, SCALED, H16ROW, 9>(a, tk, rank, smem_u, bar, phase, pending); break;
        case 10: ok = run_task<TS, MODE, SCALED, H16ROW, 10>(a, tk, rank, smem_u, bar, phase, pending); break;
        case 11: ok = run_task<TS, MODE, SCALED, H16ROW, 11>(a, tk, rank, smem_u, bar, phase, pending); break;
        case 12: ok = run_task<TS, MODE, SCALED, H16ROW, 12>(a, tk, rank, smem_u, bar, phase, pending); break;
        case 13: ok = run_task<TS, MODE, SCALED, H16ROW, 13>(a, tk, rank, smem_u, bar, phase, pending); break;
        case 14: ok = run_task<TS, MODE, SCALED, H16ROW, 14>(a, tk, rank, smem_u, bar, phase, pending); break;
        case 15: ok = run_task<TS, MODE, SCALED, H16ROW, 15>(a, tk, rank, smem_u, bar, phase, pending); break;
        case 16: ok = run_task<TS, MODE, SCALED, H16ROW, 16>(a, tk, rank, smem_u, bar, phase, pending); break;
        default: break;
      }
      aborted = !ok;
    }
    // A peer may write into this CTA's shared memory in the next task only
    // after this CTA is done with it.  Between two four-step tasks of the
    // same length with the output exchange (N1 >= 8) the data dependencies
    // already guarantee that: the CTAs that send to this one in the next task
    // are the same group, and each of them finished this task only after
    // receiving this CTA's step-3 values (sent once its row buffer was read),
    // and sends its own step-3 values of the next task only after receiving
    // this CTA's step-1 values of it (sent once its output buffer was read).
    // Every CTA of the cluster sees the same task sequence, so all skip or all
    // keep the barrier.
    const int next = task + clusters;
    const bool chained = tk.log2n >= 15 && next < a.num_tasks && a.tasks[next].log2n == tk.log2n;
    if (!chained) cluster_barrier_relaxed();
  }
  // The last task of every cluster ends with a barrier, so every peer has
  // issued all its stores by now; an aborted CTA still waits (bounded) for
  // those owed to its pending phases before its shared memory goes away.
  if (aborted) fourstep_drain(&bar[0], &bar[1], phase, pending);
}

template <class TS, int MODE, bool SCALED, bool H16ROW = false>
cudaError_t launch_typed(const UnevenArgs& a, int clusters, cudaStream_t s) {
  auto kern = uneven_kernel<TS, MODE, SCALED, H16ROW>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(clusters * kClusterCtas));
  cfg.blockDim = dim3(kCta);
  cfg.dynamicSmemBytes = uneven_smem_bytes<TS>();
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterCtas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <class TS, int MODE, bool SCALED, bool H16ROW>
cudaError_t set_attributes() {
  auto kern = uneven_kernel<TS, MODE, SCALED, H16ROW>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  if (uneven_smem_bytes<TS>() > 48 * 1024)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(uneven_smem_bytes<TS>()));
  return e;
}

// Attributes of the kernel (both exchange forms for FP16 storage, which share
// their shared memory size and so their occupancy) and its resident clusters.
template <class TS, int MODE, bool SCALED>
cudaError_t configure_typed(int* max_clusters) {
  auto kern = uneven_kernel<TS, MODE, SCALED, false>;
  cudaError_t e = set_attributes<TS, MODE, SCALED, false>();
  if (e != cudaSuccess) return e;
  if constexpr (std::is_same<TS, __half2>::value) {
    e = set_attributes<TS, MODE, SCALED, true>();
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kClusterCtas);
  cfg.blockDim = dim3(kCta);
  cfg.dynamicSmemBytes = uneven_smem_bytes<TS>();
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterCtas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(max_clusters, kern, &cfg);
}

// Storage kinds: 0 FP32, 1 FP16, 2 E4M3, 3 E5M2.
template <int MODE>
cudaError_t dispatch(int kind, bool configure, const UnevenArgs* a, int clusters, int* max_clusters,
                     cudaStream_t s) {
  using A = Fp8x2<E4M3>;
  using B = Fp8x2<E5M2>;
  switch (kind) {
    case 0: return configure ? configure_typed<float2, MODE, false>(max_clusters)
                             : launch_typed<float2, MODE, false>(*a, clusters, s);
    case 1:
      if (configure) return configure_typed<__half2, MODE, false>(max_clusters);
      return a->fs_h16 ? launch_typed<__half2, MODE, false, true>(*a, clusters, s)
                       : launch_typed<__half2, MODE, false>(*a, clusters, s);
    case 2: return configure ? configure_typed<A, MODE, true>(max_clusters)
                             : launch_typed<A, MODE, true>(*a, clusters, s);
    case 3: return configure ? configure_typed<B, MODE, true>(max_clusters)
                             : launch_typed<B, MODE, true>(*a, clusters, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t uneven_max_clusters(int kind, bool inverse, int* max_clusters) {
  return inverse ? dispatch<kInverse>(kind, true, nullptr, 0, max_clusters, nullptr)
                 : dispatch<kForward>(kind, true, nullptr, 0, max_clusters, nullptr);
}

cudaError_t launch_uneven(int kind, bool inverse, const UnevenArgs& a, int clusters, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  e = inverse ? dispatch<kInverse>(kind, false, &a, clusters, nullptr, s)
              : dispatch<kForward>(kind, false, &a, clusters, nullptr, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace bfp
