// tc_common.cuh -- fifth-generation tensor core (tcgen05) building blocks for sm_103a, as inline
// PTX: tensor-memory allocation, shared-memory matrix descriptors, the instruction descriptor of a
// BF16 x BF16 -> FP32 MMA, commit to an mbarrier, tensor-memory loads and the ordering fences.
//
// Shared-memory operands use the K-major layout without swizzle: an operand is a grid of "core
// matrices" of 8 rows x 16 bytes (8 BF16 values along K), each stored as 128 contiguous bytes
// (row r at byte 16 r).  The descriptor gives the byte distance between core matrices adjacent
// along K (leading-dimension offset) and along M or N (stride-dimension offset).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "device_common.cuh"

namespace qmmm {
namespace tc {

// 64-bit shared-memory matrix descriptor: start address, leading- and stride-dimension byte
// offsets (all in 16-byte units, 14 bits each), the fixed version field (1) of this tensor-core
// generation at bit 46, base offset 0, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;
    return d;
}

// 32-bit instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9 and
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Tensor-memory allocation (one whole warp executes these).  The allocated base address is
// written to shared memory at `dst`.  ncols: a power of two in [32, 512].
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread.  accumulate = 0 overwrites D.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The mbarrier at `bar` receives one arrival once every MMA this thread issued so far completed.
__device__ __forceinline__ void commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 8 consecutive FP32 columns of this thread's tensor-memory lane (warp w reads lanes
// 32 (w % 4) .. 32 (w % 4) + 31; taddr carries the lane in bits 16-31 and the column in 0-15).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Per-thread bounded wait for the completion of phase `parity` (no block-wide agreement: for
// warp-specialised kernels).  Gives up after `limit_ns` of global-timer time, 2^24 polls, or when
// another thread raised *abort; returns false then.  With abort == nullptr only the time and poll
// limits apply: the form for draining work already issued (bulk copies in flight, MMAs not yet
// complete) after a give-up, before the block frees what that work writes into.
__device__ __forceinline__ bool mbar_wait_thread(uint64_t *bar, unsigned parity, const volatile int *abort,
                                                 uint64_t limit_ns = MBAR_LIMIT_NS)
{
    const uint64_t t0 = global_ns();
    for (int it = 0; it < (1 << 24); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 31) == 31 && ((abort && *abort) || global_ns() - t0 > limit_ns)) return false;
    }
    return false;
}
__device__ __forceinline__ bool mbar_drain(uint64_t *bar, unsigned parity)
{
    return mbar_wait_thread(bar, parity, nullptr);
}

}  // namespace tc
}  // namespace qmmm
