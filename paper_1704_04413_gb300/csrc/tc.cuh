// 5th-generation tensor core (tcgen05) helpers for the closure network: tensor-memory (TMEM) allocation, the
// shared-memory matrix and instruction descriptors of a BF16 x BF16 -> FP32 MMA, the MMA itself (issued by one
// thread, accumulating in TMEM), its completion on an mbarrier, and TMEM loads into registers.  Inline PTX of
// the tcgen05 instruction family (PTX ISA 8.6 and later, sm_100a-family targets).
#pragma once
#include <cstdint>

#include "bulk.cuh"

namespace lbm {
namespace tc {

// Whole warp: allocate ncols TMEM columns (a power of two >= 32); the TMEM address lands in *slot (shared).
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
// Whole warp (the allocating one): release the columns.
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Order tcgen05 operations around a thread synchronisation (before it in the waiting thread's program order,
// after it in the continuing thread's).
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Make this thread's ordinary shared-memory writes visible to the tensor core's reads (the async proxy).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory matrix descriptor without swizzle: the operand is stored as core matrices of 8 rows x 16 bytes
// (128 contiguous bytes, rows 16 bytes apart), K-major (the 16 bytes of a core-matrix row run along K).
// lbo: bytes between core matrices adjacent along K; sbo: bytes between core matrices adjacent along M (or N).
// Bits: start address >> 4 [0, 14), lbo >> 4 [16, 30), sbo >> 4 [32, 46), descriptor version 1 [46, 48),
// base offset 0, layout type 0 (no swizzle) [61, 64).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3fffu);
  d |= (uint64_t)((lbo >> 4) & 0x3fffu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3fffu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16 for BF16 A and B (both K-major, dense, not negated) and an FP32
// accumulator of M x N: D format [4, 6) = 1 (FP32), A format [7, 10) = 1 (BF16), B format [10, 13) = 1 (BF16),
// N >> 3 at [17, 23), M >> 4 at [24, 29).
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// One thread: D[TMEM d] = A[smem a] x B[smem b]^T (+ D when accumulate), A M x 16, B N x 16 (BF16, K = 16).
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
      ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// The mbarrier receives one arrival once every tcgen05 MMA this thread issued before has completed.
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

// Whole warp: lane t receives TMEM lane (lane field of taddr) + t, 16 consecutive 32-bit columns from taddr's
// column.  The values are usable after wait_ld().
__device__ __forceinline__ void ld_32x32b_x16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace tc
}  // namespace lbm
