// Bulk asynchronous global -> shared copies (TMA, cp.async.bulk) completed on
// mbarriers, with bounded waits.
//
// Every wait polls at most kMaxPolls times; on expiry it records
// BFPFFT_ERR_TIMEOUT in a device status word and reports failure, so a kernel
// never spins forever on a copy that does not arrive.
#pragma once

#include <cstdint>

namespace bfp {

constexpr uint32_t kMaxPolls = 1u << 22;
constexpr unsigned long long kMaxWaitNs = 1000000000ull;   // 1 s of wall time per wait
constexpr int kStatusTimeout = 5;     // BFPFFT_ERR_TIMEOUT
constexpr int kStatusNonfinite = 6;   // BFPFFT_ERR_NONFINITE

// Output check of plans with BFPFFT_CHECK_FINITE: a thread that stored a
// non-finite value records BFPFFT_ERR_NONFINITE in the plan's status word,
// unless an earlier error is already recorded there.
__device__ __forceinline__ void note_nonfinite(int* flag, bool bad) {
  if (bad) atomicCAS(flag, 0, kStatusNonfinite);
}
// The check runs as its own loop behind `if (flag != nullptr)`, after the
// stores, so plans without the flag issue none of its instructions.  value(m)
// gives the m-th value the thread stored; S::finite says whether it is finite
// in that storage format.
template <class S, int P, class F>
__device__ __forceinline__ void check_finite(int* flag, F value) {
  if (flag == nullptr) return;
  bool bad = false;
#pragma unroll
  for (int m = 0; m < P; ++m) bad |= !S::finite(value(m));
  note_nonfinite(flag, bad);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make barrier initialisation and prior generic-proxy shared accesses visible
// to the async (TMA) proxy.
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// 1-D bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of `bar`; false (and status set) on expiry.
// A try_wait may suspend the thread for a while, so the bound is wall time
// (kMaxWaitNs) as well as a poll count.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (uint32_t i = 0; i < kMaxPolls; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 63u && global_ns() - t0 > kMaxWaitNs) break;
  }
  if (status != nullptr) atomicExch(status, kStatusTimeout);
  return false;
}

// Bulk prefetch of [p, p + bytes) into L2 (p 16-byte aligned, bytes a multiple
// of 16); no completion to wait for.
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}

// Asynchronous store of one complex FP32 value into another CTA's shared
// memory; its arrival is counted (8 bytes) on that CTA's mbarrier.
__device__ __forceinline__ void st_async_f2(uint32_t remote_addr, float2 v, uint32_t remote_bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(remote_addr),
               "f"(v.x), "f"(v.y), "r"(remote_bar)
               : "memory");
}

__device__ __forceinline__ void st_async_b32(uint32_t remote_addr, uint32_t v, uint32_t remote_bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(remote_addr), "r"(v),
               "r"(remote_bar)
               : "memory");
}

// 32-bit loads and stores of shared::cluster addresses (from mapa).
__device__ __forceinline__ uint32_t ld_cluster_b32(uint32_t addr) {
  uint32_t r;
  asm volatile("ld.shared::cluster.b32 %0, [%1];" : "=r"(r) : "r"(addr) : "memory");
  return r;
}
__device__ __forceinline__ void st_cluster_b32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared::cluster.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// Split cluster barrier halves (non-aligned forms).
__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
  asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}

// Cluster barrier without memory ordering (only "everyone got here").
__device__ __forceinline__ void cluster_barrier_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed;\n\tbarrier.cluster.wait;" ::: "memory");
}

}  // namespace bfp
