// staging.cuh -- TMA bulk copies of CSR slices into shared memory, with an
// mbarrier per stage and bounded waits.
//
// A persistent block walks tiles of consecutive rows.  While it computes tile
// t from one shared-memory stage, one thread has already issued the bulk
// copies (cp.async.bulk, the Tensor Memory Accelerator's 1-D mode) of tile
// t+grid's column indices and values into the other stage; completion is
// tracked by the stage's mbarrier (transaction bytes).  A bulk copy needs a
// 16-byte aligned source, destination and size: the slice [s0, s1) is
// widened to [s0a, s1a) on 16-byte boundaries (the arrays are allocated with
// 16 bytes of padding), and entries are addressed relative to s0a.
//
// Every wait is bounded: after `limit` clock cycles the waiting thread sets
// the handle's device status word and gives up (the caller then leaves the
// kernel); no wait can spin forever.
#pragma once

#include <stdint.h>

namespace amgd {

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// make the barrier initialisation visible to the async (TMA) proxy
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order earlier generic-proxy accesses of shared memory before later
// async-proxy writes to it (a stage is refilled after it was read)
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared, completion reported to `bar`
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// wait for phase `parity` of `bar` for at most `limit` cycles; on time-out
// set `status` (bit value `code`) and return false
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit,
                                                  uint32_t *status, uint32_t code)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) {
            atomicOr(status, code);
            return false;
        }
    }
    return true;
}

// 16-byte asynchronous copy global -> shared (lands without holding
// registers; completion per thread through commit/wait groups)
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace amgd
