// Fifth-generation tensor-core helpers (sm_103a): tcgen05 MMA with BF16
// operands in shared memory and FP32 accumulators in tensor memory (TMEM),
// issued by one thread and tracked by an mbarrier.  Used by the
// level-of-detail network's kernels (kl_mlp.cu).
//
// Operand tiles are stored K-major without swizzling, as 8-row x 16-byte
// core matrices: element (r, k) of a BF16 tile lies at
//     (r / 8) * SBO + (k / 8) * LBO + (r % 8) * 16 + (k % 8) * 2,
// SBO = 128 bytes (the eight rows of a core matrix back to back, then the
// next eight rows), LBO = the distance between the 8-element K chunks.  One
// kind::f16 MMA consumes 16 K elements (two chunks), so successive K steps
// advance the start address by 2 LBO.
#pragma once

#include <stdint.h>

namespace {

constexpr uint32_t kTcSBO = 128;

__host__ __device__ constexpr uint32_t tc_off(uint32_t r, uint32_t k, uint32_t lbo) {
  return (r / 8) * kTcSBO + (k / 8) * lbo + (r % 8) * 16 + (k % 8) * 2;
}

// The same tile stored MN-major: the 8 MN elements of a core matrix row are
// contiguous (16 bytes) and its 8 K values lie 16 bytes apart.  Element
// (r, k) at (r / 8) * SBO + (k / 8) * LBO + (k % 8) * 16 + (r % 8) * 2; the
// descriptor takes LBO and SBO in the same roles, and the instruction
// descriptor marks the operand MN-major.  A thread owning one K index (a
// row of the batch) writes 8 consecutive MN elements with one 16-byte store.
__host__ __device__ constexpr uint32_t tc_off_mn(uint32_t r, uint32_t k, uint32_t lbo) {
  return (r / 8) * kTcSBO + (k / 8) * lbo + (k % 8) * 16 + (r % 8) * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, LBO and SBO in 16-byte
// units, descriptor version 1 (bits 46-47), no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(kTcSBO >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 and 10-12 = 1), A and B K-major (bits 15, 16 = 0) or
// MN-major (= 1), N / 8 in bits 17-22, M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(uint32_t M, uint32_t N, uint32_t a_mn = 0,
                                                     uint32_t b_mn = 0) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (a_mn << 15) | (b_mn << 16) | ((N >> 3) << 17) |
         ((M >> 4) << 24);
}

// TMEM columns [0, ncols) for this CTA (one full warp calls it); the address
// is written to *slot.  ncols: a power of two >= 32.
__device__ __forceinline__ void tc_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// D (TMEM) = A B (acc = 0) or D += A B (acc != 0); M = 128 rows of A.
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// The mbarrier completes one phase when every MMA this thread issued before
// has finished.
__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar))
      : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait for the phase of the given parity to complete, for at most
// `limit` clock cycles; false if it did not.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Make this thread's ordinary shared-memory stores visible to the tensor
// cores (the async proxy) before an MMA reads them.
__device__ __forceinline__ void fence_smem_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (warp w of the CTA
// reads lanes 32 w .. 32 w + 31; taddr carries the lane in bits 16-31).
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

}  // namespace
