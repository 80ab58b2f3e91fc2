// fh_tma.cuh -- bulk asynchronous copies (the TMA engine's 1-D form) between
// global and shared memory, completed through shared-memory mbarriers.
//
// Rules these helpers rely on (PTX ISA, cp.async.bulk):
//  * global and shared addresses 16-byte aligned, size a multiple of 16;
//  * a load signals completion by complete_tx on an mbarrier whose expected
//    transaction count was raised by the same number of bytes;
//  * shared memory written by ordinary stores must be fenced into the async
//    proxy (fence.proxy.async.shared::cta) before a bulk store reads it;
//  * a buffer read by a bulk store may be overwritten only after
//    cp.async.bulk.wait_group.read has returned in the issuing thread.
// Every wait is bounded by a wall-clock limit so that a lost completion ends
// the kernel with an error word instead of a hang.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fh {
namespace tma {

// Default limit of one wait.  Kernels take their primary waits' limit from
// their launch arguments (fh_set_wait_limit; 0 there means this default); the
// waits that drain a kernel's own copies in flight after a failure always use
// this default, so that no copy can land in shared memory the kernel has left.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per wait

// Process-wide limit set by fh_set_wait_limit (host side; 0 = default).
unsigned long long wait_limit_ns();

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

// Make initialised barriers visible to the async proxy.
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Order this thread's generic-proxy shared-memory writes before later
// async-proxy accesses (bulk stores that read them).
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)),
               "r"(bytes)
               : "memory");
}

// global -> shared, completion counted on bar
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          saddr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(saddr(bar))
      : "memory");
}

// shared -> global, tracked by the issuing thread's bulk groups
__device__ __forceinline__ void bulk_store(void* dst_gmem, const void* src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
               "r"(saddr(src_smem)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// the shared-memory sources of every committed bulk store have been read
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// every committed bulk store has completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Wait until phase `parity` of bar has completed; false after limit_ns
// nanoseconds (0: kWaitLimitNs).  try_wait may suspend the thread for a
// hardware-chosen time while the phase is incomplete; with an explicit limit
// that suspension is capped by the limit itself (the instruction's
// suspend-time hint), so a short limit runs out even while a copy is still
// in flight.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long limit_ns = 0) {
  const uint32_t a = saddr(bar);
  const unsigned long long t0 = globaltimer();
  if (limit_ns == 0) {
    while (true) {
      uint32_t ok;
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(ok)
          : "r"(a), "r"(parity)
          : "memory");
      if (ok) return true;
      if (globaltimer() - t0 > kWaitLimitNs) return false;
    }
  }
  const uint32_t hint = limit_ns < 0x7fffffffull ? (uint32_t)limit_ns : 0x7fffffffu;
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity), "r"(hint)
        : "memory");
    if (ok) return true;
    if (globaltimer() - t0 > limit_ns) return false;
  }
}

}  // namespace tma
}  // namespace fh
