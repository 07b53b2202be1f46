// Fifth-generation tensor-core (tcgen05) building blocks for the quantised
// tile products: shared-memory matrix descriptors, the instruction
// descriptor, the MMA, its commit to an mbarrier, and the tensor-memory
// (TMEM) allocation and loads.  All inline PTX for sm_100-family GPUs.
//
// Operand layout ("no swizzle" canonical layout): a matrix is cut into core
// matrices of 8 rows x 16 bytes, each stored as 128 contiguous bytes (row i
// of the core at byte 16 i).  A descriptor gives the start address and two
// strides between core matrices:
//   K-major operand (rows = M or N, 16-byte rows along K):
//     LBO = stride between cores along K, SBO = stride along M / N;
//   MN-major operand (16-byte rows along M, 8 rows along K):
//     LBO = stride between cores along K, SBO = stride along M.
// One stored tile in this layout serves both as A (K-major, the product
// Q d) and as A' = Q' (MN-major, the product Q' d), which is how a single
// read of a symmetric-matrix tile feeds both of its products.
#pragma once

#include <cstdint>

namespace rapdb_dev {

// Shared-memory matrix descriptor (sm_100 family): start address, LBO and
// SBO in 16-byte units (bits 0-13, 16-29, 32-45), descriptor version 1
// (bits 46-47), base offset 0, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t umma_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of a dense MMA with float32 accumulation:
// bits 4-5 D format (1 = f32); bits 7-9 / 10-12 A / B format (kind::f16:
// 1 = bf16; kind::f8f6f4: 0 = e4m3); bit 15 A MN-major; bit 16 B MN-major;
// bits 17-22 N >> 3; bits 24-28 M >> 4.
__host__ __device__ constexpr uint32_t umma_idesc(bool f8, bool a_mn_major, uint32_t M, uint32_t N) {
  return (1u << 4) | ((f8 ? 0u : 1u) << 7) | ((f8 ? 0u : 1u) << 10) | ((a_mn_major ? 1u : 0u) << 15) |
         ((N >> 3) << 17) | ((M >> 4) << 24);
}

// D[tmem] (+)= A * B, issued by one thread; acc = 0 overwrites D.
template <bool F8>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                     uint32_t acc) {
  if constexpr (F8) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(acc)
        : "memory");
  }
}

// The mbarrier receives one arrival when every MMA this thread issued before
// has completed (its shared-memory operands read, its D written).
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// One lane of a converged warp (the lowest active one).  The MMA and copy
// loops run on whole warps, so that their addresses and descriptors stay
// warp-uniform, and the elected lane issues: a loop run by one lane alone
// issued an MMA every ~85 cycles, a whole warp every ~39 (measured, 128 x 16
// x 16 BF16 MMAs).
__device__ __forceinline__ bool elect_one() {
  uint32_t pred = 0;
  asm volatile("{\n .reg .pred p;\n elect.sync _|p, 0xffffffff;\n selp.u32 %0, 1, 0, p;\n}\n" : "=r"(pred));
  return pred != 0;
}

// Ordering of tensor-core operations around thread barriers.
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TMEM allocation by one whole warp: the base address is written to *slot.
// One CTA per SM uses TMEM here, so the allocation never waits.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Eight consecutive 32-bit TMEM columns of this thread's lane (the warp
// reads lanes 32 (warp % 4) .. + 31; taddr carries the lane base in bits
// 16-31).  The wait is in the same statement, so no use of v can move
// above it.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace rapdb_dev
