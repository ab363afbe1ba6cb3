// tcgen05.cuh -- inline-PTX helpers for the fifth-generation tensor cores
// (tcgen05.mma with TMEM accumulators), mbarriers and named barriers, shared
// by the digit-product kernels of the per-frequency matrix products.
//
// Shared-memory operand layout (no swizzle).  The unit is the "core matrix"
// of 8 rows x 16 bytes.  A K-major tile (B operand: rows n, 8 consecutive k in
// 16 bytes) and an MN-major tile (A operand: 8 consecutive m in 16 bytes, one
// row per k) both place the next group of 8 k at +128 bytes (the leading
// byte offset) and the next group of 8 rows of M or N at +SBO bytes (the
// stride byte offset).  These encodings were checked on the GPU against exact
// integer GEMMs before the product kernels were built on them.
#pragma once
#include <stdint.h>

namespace mrc_tc {

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address >> 4, leading byte offset
// 128 >> 4 at bit 16, stride byte offset SBO >> 4 at bit 32, the fixed
// 0b001 at bits 46-48, no swizzle.
template <int SBO>
__device__ __forceinline__ uint64_t desc(unsigned addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(SBO >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9, 10-12 = 1), A MN-major (bit 15), B K-major, N >> 3 at bit 17,
// M >> 4 at bit 24.
template <int M, int N>
constexpr unsigned idesc_bf16() { return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24); }

// D (TMEM) (+)= A (smem) . B (smem); acc = 0 overwrites D
template <unsigned IDESC>
__device__ __forceinline__ void mma(unsigned dtm, uint64_t ad, uint64_t bd, unsigned acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
                 "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
                 : "memory");
}

// arrive once on the mbarrier when every tcgen05 operation this thread issued so far has completed
__device__ __forceinline__ void commit(unsigned mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the tensor cores (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(unsigned mbar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(unsigned mbar)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}

// Bounded wait for the completion of phase `parity` of an mbarrier: at most
// `spins` rounds of try_wait, each suspending the thread for at most about
// SUSPEND_NS nanoseconds.  Returns false if the wait gave up.
constexpr unsigned SUSPEND_NS = 1000;
constexpr int SPIN = 1 << 22;
__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity, int spins = SPIN)
{
    for (int it = 0; it < spins; ++it) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity), "r"(SUSPEND_NS)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// One arrival on the mbarrier that also expects `bytes` of asynchronous
// copies to complete on it in the current phase
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned mbar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes)
                 : "memory");
}

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global memory into this CTA's shared memory, completing as
// transaction bytes on the mbarrier
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void *src, unsigned bytes, unsigned mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

// Bulk prefetch of `bytes` (a multiple of 16, 16-byte aligned) of global
// memory into L2, without a destination in shared memory
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// Named barrier over `count` threads (a multiple of 32); the OR of `pred`
// over them is returned to every one.
__device__ __forceinline__ bool bar_or(int id, int count, bool pred)
{
    unsigned r;
    asm volatile("{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n"
                 " barrier.cta.red.or.pred po, %2, %3, pi;\n selp.u32 %0, 1, 0, po;\n}\n"
                 : "=r"(r)
                 : "r"((unsigned)pred), "r"(id), "r"(count)
                 : "memory");
    return r != 0;
}
__device__ __forceinline__ void bar_sync(int id, int count)
{
    asm volatile("barrier.cta.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}

// TMEM allocation by one whole warp (columns: a power of two >= 32)
__device__ __forceinline__ void tmem_alloc(unsigned slot_smem, unsigned cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot_smem), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(cols) : "memory");
}

// 32 TMEM lanes x 8 consecutive 32-bit columns: thread `lane` of the warp
// receives lane (base lane + lane), columns col .. col + 7; then waits.
__device__ __forceinline__ void ld8(unsigned taddr, unsigned (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// BF16 bits of two exact small integers (|q| <= 256 has at most 8
// significant bits, so the high half of the binary32 is the BF16 value),
// packed low | high
__device__ __forceinline__ unsigned pack2(float lo, float hi)
{
    return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

} // namespace mrc_tc
