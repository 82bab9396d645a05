// 1-D bulk copies global -> shared through the tensor memory accelerator
// (cp.async.bulk with an mbarrier transaction count), with bounded waits.
//
// Rules kept by every caller: source and destination 16-byte aligned, size a
// multiple of 16 bytes; the barrier is initialised by one thread and made visible
// to the async proxy before the first copy; a buffer is refilled only after a
// block-wide barrier following its last read (plus a proxy fence).  Every wait
// gives up after a fixed number of polls, so a lost transfer turns into an error
// status instead of a hang.
#pragma once

#include <stdint.h>

namespace qnep {

constexpr uint32_t kWaitPolls = 1u << 22;   // bounded mbarrier wait (far above any real transfer time)
constexpr unsigned kStatusTimeout = 2u;     // Accum::status bit set when a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make barrier initialisation visible to the async proxy
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order earlier generic-proxy accesses of shared memory before later async-proxy writes
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// the same for global and shared memory: data the block wrote with ordinary stores (after a
// block barrier) is then read correctly by a following bulk copy
__device__ __forceinline__ void fence_proxy_async_all() {
    asm volatile("fence.proxy.async;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// one arrival without a transaction count (completes a phase of a count-1 barrier)
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the barrier to complete; false after kWaitPolls polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (uint32_t it = 0; it < kWaitPolls; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__host__ __device__ constexpr uint32_t round_up16(uint32_t b) { return (b + 15u) & ~15u; }

}  // namespace qnep
