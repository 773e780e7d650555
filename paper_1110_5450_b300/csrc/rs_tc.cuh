// rs_tc.cuh -- fifth-generation tensor-core (tcgen05) building blocks for
// sm_103a: tensor-memory allocation, BF16/FP16 MMAs with FP32 accumulators in
// tensor memory, completion through an mbarrier, and accumulator loads.
//
// Operands live in shared memory in the canonical no-swizzle layout: "core
// matrices" of 8 rows x 16 bytes (8 rows x 8 16-bit elements).  For an
// operand with the reduction dimension K contiguous (K-major) the 16 bytes of
// a core-matrix row run along K; for an MN-major operand they run along M (or
// N).  A 64-bit shared-memory descriptor gives the start address and the byte
// distances between neighbouring core matrices in the two directions.
#pragma once

#include <stdint.h>

namespace rs {
namespace tc {

__device__ __forceinline__ uint32_t saddr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address, leading- and
// stride-dimension byte offsets (all >> 4), descriptor version 1, no swizzle.
__host__ __device__ inline uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= uint64_t((addr >> 4) & 0x3FFFu);
    d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
    d |= uint64_t(1) << 46; // descriptor version
    return d;
}

// The same for a K-major operand in the 128-byte swizzled layout (rows of 128
// bytes of K, 16-byte chunks permuted by row % 8 as a TMA copy with
// CU_TENSOR_MAP_SWIZZLE_128B lands them, from a 1024-byte aligned base): sbo =
// distance between groups of 8 rows; the leading offset is unused; advancing
// K within a row adds to the start address.
__host__ __device__ inline uint64_t smem_desc_sw128(uint32_t addr, uint32_t sbo)
{
    uint64_t d = smem_desc(addr, 16u, sbo);
    d |= uint64_t(2) << 61; // swizzling mode: 128-byte
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulators, A and B of the
// same 16-bit type (bf16 = true: BF16, else FP16), major-ness of A and B
// (1 = MN-major), shape M x N.
__host__ __device__ inline uint32_t idesc_f16(bool bf16, bool a_mn, bool b_mn, int M, int N)
{
    uint32_t d = 0;
    d |= 1u << 4;                       // D format: FP32
    d |= (bf16 ? 1u : 0u) << 7;         // A format
    d |= (bf16 ? 1u : 0u) << 10;        // B format
    d |= (a_mn ? 1u : 0u) << 15;        // A major
    d |= (b_mn ? 1u : 0u) << 16;        // B major
    d |= uint32_t(N >> 3) << 17;        // N / 8
    d |= uint32_t(M >> 4) << 24;        // M / 16
    return d;
}

// Tensor-memory allocation (one full warp).  The base address is written to
// *slot (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D(tmem) (+)= A(smem) * B(smem); issued by a single thread.
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on an mbarrier once all previously issued MMAs of this thread complete.
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Generic-proxy shared-memory writes made visible to the tensor cores.
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 16 consecutive 32-bit accumulator columns of this thread's lane
// (warp w of a 128-thread group reads lanes 32w .. 32w + 31).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_ld_wait()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Byte offset of element (r, k) of an operand in the canonical no-swizzle
// layout.  K-major: core matrices are 8 rows x 8 k; stride_k is the distance
// between core matrices along K, stride_r between 8-row groups.  MN-major:
// core matrices are 8 k x 8 rows (16 bytes along the rows).
__host__ __device__ inline uint32_t canon_offset(bool mn_major, int r, int k, uint32_t stride_r, uint32_t stride_k)
{
    if (!mn_major) return uint32_t(r / 8) * stride_r + uint32_t(k / 8) * stride_k + uint32_t(r % 8) * 16 + uint32_t(k % 8) * 2;
    return uint32_t(r / 8) * stride_r + uint32_t(k / 8) * stride_k + uint32_t(k % 8) * 16 + uint32_t(r % 8) * 2;
}

} // namespace tc
} // namespace rs
