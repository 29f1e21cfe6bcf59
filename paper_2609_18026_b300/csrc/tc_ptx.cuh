// Inline-PTX helpers shared by the tensor-core kernels of libmlx (the Legendre
// contraction and the surrogate's GEMM): shared-memory addresses, mbarriers with
// bounded waits, TMA tile loads, tcgen05 MMA / commit / TMEM load, and the
// shared-memory matrix descriptors of K-major operands.
#pragma once

#include <stdint.h>

namespace tcx {

constexpr long long kSpinLimit = 1LL << 22;   // try_wait polls before a wait gives up

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of the given parity to complete, at most kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  for (long long it = 0; it < kSpinLimit; ++it)
    if (mbar_try(bar, parity)) return true;
  return false;
}
// The same, giving up early when *abort becomes nonzero (another role gave up).
__device__ __forceinline__ bool mbar_wait_or_abort(unsigned bar, unsigned parity, volatile int* abort) {
  for (long long it = 0; it < kSpinLimit; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 63) == 63 && *abort) return false;
  }
  return false;
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// make this thread's generic-proxy shared-memory writes visible to the async proxy
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 3-D tiled TMA load into shared memory, completion counted on an mbarrier
__device__ __forceinline__ void tma_load_3d(unsigned dst, const void* tmap, int c0, int c1, int c2, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_2d(unsigned dst, const void* tmap, int c0, int c1, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(tmap), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

// Tensor memory: allocation by one warp (power of two >= 32 columns)
__device__ __forceinline__ void tmem_alloc(unsigned slot_smem, unsigned cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_smem), "r"(cols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(unsigned tmem, unsigned cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D (TMEM, FP32) (+)= A (smem) * B (smem)^T, BF16 operands, one elected thread
__device__ __forceinline__ void mma_bf16(unsigned tmem, uint64_t da, uint64_t db, unsigned idesc, unsigned acc) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }"
      ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}
// arrive on an mbarrier once every MMA this thread issued before has completed
__device__ __forceinline__ void mma_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major
__device__ __forceinline__ unsigned idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

// 32 lanes x 32 bits, 16 consecutive columns of this warp's TMEM lane quarter
__device__ __forceinline__ void tmem_ld16(unsigned taddr, unsigned (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory descriptors of K-major operands (start address, leading byte
// offset 16, stride between 8-row groups, descriptor version 1, swizzle mode).
// 128-byte swizzle: rows of 128 bytes (64 BF16), 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(unsigned saddr) {
  return ((uint64_t)((saddr >> 4) & 0x3FFF)) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// 64-byte swizzle: rows of 64 bytes (32 BF16), 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t desc_sw64(unsigned saddr) {
  return ((uint64_t)((saddr >> 4) & 0x3FFF)) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}
// byte offset of element k (BF16) of row `row` in the 128-byte-swizzled layout
__device__ __forceinline__ unsigned sw128_offset(int row, int k) {
  return (unsigned)(row * 128 + ((((k >> 3) ^ (row & 7)) & 7) << 4) + ((k & 7) << 1));
}
// ... and in the 64-byte-swizzled layout: the 16-byte chunk index XOR bits 1-2 of
// the row (the pattern repeats every 8 rows = 512 bytes)
__device__ __forceinline__ unsigned sw64_offset(int row, int k) {
  return (unsigned)(row * 64 + ((((k >> 3) ^ (row >> 1)) & 3) << 4) + ((k & 7) << 1));
}

}  // namespace tcx
