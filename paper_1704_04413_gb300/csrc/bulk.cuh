// Asynchronous bulk copies global -> shared (cp.async.bulk, the TMA unit's untiled form) completing on
// shared-memory mbarriers, for the staged step kernels.  Every wait is bounded by a time limit on the global
// nanosecond timer; callers turn a wait that gives up into an error word and return instead of spinning.
#pragma once
#include <cstdint>

namespace lbm {

constexpr unsigned long long kBulkWaitNs = 1000000000ull;  // 1 s: a wait on a copy that never completes

// Run-time control of a staged kernel's waits, passed by value.
struct StageCtl {
  int* status;                 // device word: set when a bounded wait gave up
  unsigned long long wait_ns;  // limit of every bounded wait (kBulkWaitNs unless a test shortens it)
  int fault_block;             // test hook: this block's producer announces but never issues the copies of
                               // its last tile, so its compute warps' wait runs out; -1: off
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes the initialised barriers visible to the async proxy (the copies that complete on them).
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival that also announces `bytes` of copies completing on this phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// One plain arrival (no transaction bytes).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// dst (shared) <- src (global), `bytes` a nonzero multiple of 16, both addresses 16-byte aligned.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Suspends the thread until the phase of parity `parity` completes or about kBulkSuspendNs pass (a waiting
// warp sleeps instead of taking issue slots from the warps that compute).
constexpr uint32_t kBulkSuspendNs = 1000000u;

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(kBulkSuspendNs)
      : "memory");
  return ok != 0;
}

// Waits until the phase of parity `parity` has completed; false after limit_ns without it.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long limit_ns = kBulkWaitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}

}  // namespace lbm
