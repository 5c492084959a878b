// Blackwell (sm_103a) primitives of the FP32 Gram-Schmidt and restart tiles: bulk tensor
// copies (TMA) with 32-byte swizzle, tcgen05.mma kind::tf32 with shared-memory operand
// descriptors and accumulators in tensor memory (TMEM), and the mbarriers that order them.
//
// Operand layout (K-major, 32-byte swizzle).  An operand is built from 256-byte atoms of
// 8 rows x 32 bytes (8 FP32 values along K); inside an atom the two 16-byte halves of rows
// 4..7 are swapped, i.e. value (row m, k) sits at byte 32 m + 16 ((k / 4) ^ ((m / 4) % 2))
// + 4 (k % 4) of a 256-byte-aligned atom.  Consecutive 8-row groups along M (or N) are
// SBO bytes apart; one MMA consumes K = 8 values, exactly one atom width.  A tile of 128
// rows of one basis block (n x 8 row-major in HBM) loaded by a TMA copy with 32-byte
// swizzle is therefore, as it lands, the K-major operand of Q H (M = 128 rows, K = the
// block's 8 columns) with SBO = 256.
//
// TF32 arithmetic: the tensor core reads the top 19 bits of an FP32 operand (it truncates),
// so an FP32 value x is split into hi = x with its 13 low mantissa bits cleared (the raw
// value serves as hi) and lo = x - hi (exact in FP32) rounded to the nearest tf32; a
// product is formed as hi*hi + hi*lo + lo*hi (+ lo*lo where it comes for free), about
// 2^-21 relative: the accuracy of FP32.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace usbs {
namespace tc {

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count));
}
__device__ __forceinline__ void bar_inval(uint64_t* b) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(su32(b)));
}
__device__ __forceinline__ void bar_expect_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_test(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on one phase of an mbarrier: try_wait suspends the thread until the phase
// completes or about 1 us passes; at most 2^17 tries (about 0.13 s).  False if the phase
// did not complete.
__device__ __forceinline__ bool bar_wait(uint64_t* b, unsigned parity) {
  for (int k = 0; k < (1 << 17); ++k) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity), "r"(1000u)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// 128 rows x 8 FP32 of block `blk` starting at row `row0`, from a 3-D tensor map
// {8 values, n rows, blocks}; rows past n arrive as zeros.
__device__ __forceinline__ void tma_tile(void* dst, const CUtensorMap* map, int row0, int blk, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(su32(dst)), "l"(map), "r"(0), "r"(row0), "r"(blk), "r"(su32(bar))
      : "memory");
}

// shared-memory operand descriptor: K-major, 32-byte swizzle, 8-row groups SBO bytes apart
__device__ __forceinline__ uint64_t desc_k32(uint32_t saddr, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)6 << 61);
}
// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
// arrive on *bar once every MMA issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, int ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, int ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the tensor core and to TMA
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane (the warp reads lanes
// 32 (warp % 4) .. + 31; taddr carries the lane base in its upper 16 bits)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// float index of (row m, k) inside a 256-byte atom (or a 32-byte-row swizzled tile)
__device__ __forceinline__ int sw(int m, int k) { return m * 8 + ((((k >> 2) ^ ((m >> 2) & 1)) << 2) | (k & 3)); }

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }
// x - hi(x), rounded to the nearest tf32 (so that the tensor core's truncation keeps it)
__device__ __forceinline__ float tf32_lo(float x, float hi) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x - hi));
  return __uint_as_float(r);
}

// 4 consecutive accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc
}  // namespace usbs
