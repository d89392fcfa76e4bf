// bulk.cuh -- 1-D bulk asynchronous copies (the TMA unit) from global into
// shared memory, completed on an mbarrier in shared memory, with waits that
// give up after a bounded number of polls.
//
// Use: one thread initialises the barriers (count 1) and fences the
// initialisation; a copy is armed and issued by one thread (bulk_load: the
// barrier expects the bytes, the copy completes them); every consumer polls
// the barrier's phase parity. A stage is refilled only after a block barrier
// that follows the last read of it, with fence_async_smem() before the new
// copy (generic-proxy reads ordered before the async-proxy write).
// Requirements of the hardware: source and destination 16-byte aligned, the
// size a multiple of 16 bytes.
#pragma once

#include <cstdint>

namespace rbf {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes barrier initialisations visible to the async proxy (before the block
// barrier that publishes them).
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Orders this thread's earlier shared-memory accesses before later
// async-proxy writes (a refill of a stage that was read).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Arms `bar` for `bytes` and copies [src, src + bytes) to dst.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Non-blocking test of the phase with the given parity.
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Polls the phase at most `limit` times (short sleeps after the first 64);
// false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long limit)
{
    for (unsigned long long i = 0; i < limit; ++i) {
        if (mbar_test(bar, parity)) return true;
        if (i >= 64) __nanosleep(64);
    }
    return false;
}

}  // namespace rbf
