// Bulk tensor copies (TMA) between the state in HBM and shared memory, and the
// mbarrier that signals their completion, as inline PTX for sm_103a.
//
// Loads complete on an mbarrier (expected byte count armed by one thread);
// stores are tracked in per-thread bulk groups.  Every wait is bounded by the
// global timer: a kernel whose wait gives up records kWaitTimeout in its
// translation unit's device status word and returns; the host reads the
// word in sv_sync.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace sv {

constexpr unsigned kWaitTimeout = 1u;
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// one arrival that also adds `bytes` to the transaction count of the phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// one plain arrival (a consumer releasing a buffer)
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase of the given parity to complete, for at most
// kWaitLimitNs; false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > kWaitLimitNs) return false;
  return true;
}

// generic-proxy shared-memory writes -> visible to the async proxy (TMA)
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// global -> shared, rank 2..5, coordinates c[0..rank)
template <int RANK>
__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* map, const int* c,
                                         uint32_t bar) {
  const uint64_t m = reinterpret_cast<uint64_t>(map);
  if constexpr (RANK == 2)
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(m), "r"(c[0]), "r"(c[1]), "r"(bar)
        : "memory");
  else if constexpr (RANK == 3)
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(bar)
        : "memory");
  else if constexpr (RANK == 4)
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(bar)
        : "memory");
  else
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
        "l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(bar)
        : "memory");
}

// global -> L2 only, rank 2..5: a hint that brings a box into L2 ahead of
// its load (no completion to wait for)
template <int RANK>
__device__ __forceinline__ void tma_prefetch(const CUtensorMap* map, const int* c) {
  const uint64_t m = reinterpret_cast<uint64_t>(map);
  if constexpr (RANK == 2)
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];"
                 ::"l"(m), "r"(c[0]), "r"(c[1]) : "memory");
  else if constexpr (RANK == 3)
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];"
                 ::"l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]) : "memory");
  else if constexpr (RANK == 4)
    asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];"
                 ::"l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]) : "memory");
  else
    asm volatile("cp.async.bulk.prefetch.tensor.5d.L2.global.tile [%0, {%1, %2, %3, %4, %5}];"
                 ::"l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]) : "memory");
}

// shared -> global, rank 2..5, tracked in the calling thread's bulk group
template <int RANK>
__device__ __forceinline__ void tma_store(const CUtensorMap* map, const int* c, uint32_t src) {
  const uint64_t m = reinterpret_cast<uint64_t>(map);
  if constexpr (RANK == 2)
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];"
                 ::"l"(m), "r"(c[0]), "r"(c[1]), "r"(src)
                 : "memory");
  else if constexpr (RANK == 3)
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];"
        ::"l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(src)
        : "memory");
  else if constexpr (RANK == 4)
    asm volatile(
        "cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];"
        ::"l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(src)
        : "memory");
  else
    asm volatile(
        "cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group"
        " [%0, {%1, %2, %3, %4, %5}], [%6];" ::"l"(m),
        "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(src)
        : "memory");
}

__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// this thread's committed bulk stores have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// this thread's committed bulk stores are complete
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

}  // namespace sv
