// zm_tc.cuh -- inline-PTX wrappers for the fifth-generation tensor cores of sm_100-family GPUs
// (tcgen05: tensor memory allocation, tensor memory -> register loads, MMA with both operands in
// shared memory and the accumulator in tensor memory, completion through mbarriers), used by the
// FP32C Birkhoff-Rott kernel's tensor-core far path (zm_br32tc.cu).
//
// Tensor memory (TMEM) is 512 columns x 128 lanes of 32-bit cells per SM.  An address is
// (lane << 16) | column.  Warp w of a CTA may move data only in lanes 32 (w % 4) .. + 31.
#pragma once

#include <stdint.h>

#include "zm_internal.cuh"

namespace zm {
namespace tc {

// ---- allocation (one full warp executes these) -------------------------------------------------
__device__ __forceinline__ void alloc(uint32_t *smem_dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     dev::smem_u32(smem_dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// ---- ordering of tensor-memory operations around thread synchronisation ---------------------
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ---- tensor memory -> registers (warp-collective) ------------------------------------------
// v[0..15] <- 16 consecutive columns of this thread's lane
__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t v[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---- MMA (issued by one thread) -------------------------------------------------------------------
// Shared-memory matrix descriptor, no swizzling: the matrix is a grid of core matrices of 8 rows
// x 16 bytes (each 128 contiguous bytes, rows 16 bytes apart); lbo = byte distance between core
// matrices adjacent along K (0 reads one core matrix twice), sbo = along M/N.  Bits 46-48 hold
// the fixed descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(const void *smem, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((dev::smem_u32(smem) >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32 with FP32 accumulation, A and B K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n)
{
    return (1u << 4)                           // D: FP32
           | (2u << 7) | (2u << 10)            // A, B: TF32
           | ((uint32_t)(n >> 3) << 17)        // N / 8
           | ((uint32_t)(m >> 4) << 24);       // M / 16
}

// D[tmem] (+)= A[smem desc] * B[smem desc]; accumulate = false overwrites D.
__device__ __forceinline__ void mma_tf32_ss(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                            bool accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

// The mbarrier receives one arrival when every MMA this thread issued before has completed.
__device__ __forceinline__ void commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     dev::smem_u32(bar))
                 : "memory");
}

}  // namespace tc
}  // namespace zm
