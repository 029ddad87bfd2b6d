// Inline-PTX helpers of the kernels that stream through a ring of
// shared-memory slots filled by bulk asynchronous copies (cp.async.bulk,
// completion counted on mbarriers).  Every wait is bounded.
#pragma once
#include <cstdint>

constexpr unsigned SW_WAIT = 1u << 22;   // mbarrier polls before a wait gives up

__device__ __forceinline__ void sw_mb_init(uint32_t a, unsigned c)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(c) : "memory");
}
__device__ __forceinline__ void sw_mb_expect(uint32_t a, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void sw_mb_arrive(uint32_t a)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool sw_mb_wait(uint32_t a, unsigned parity)
{
    for (unsigned it = 0; it < SW_WAIT; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void sw_bulk_g2s(uint32_t dst, const void *src, unsigned bytes, uint32_t mb)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mb)
                 : "memory");
}
// bulk prefetch of global memory into L2 (no completion, no shared memory)
__device__ __forceinline__ void sw_prefetch_l2(const void *src, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
