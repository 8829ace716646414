// Shared-memory mbarrier helpers (sm_90+ PTX) with bounded waits: a wait
// gives up after a fixed number of polls so that a kernel never spins
// forever; the caller records the timeout in the step's status flag.
#pragma once

#include <stdint.h>

namespace lbmk {

constexpr unsigned int kFlagNonfinite = 1u;
constexpr unsigned int kFlagTimeout = 2u;
constexpr long long kMbarSpinLimit = 1LL << 22;  // polls before a wait gives up (~0.1 s; copies take microseconds)

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(a), "r"(bytes) : "memory");
}
// one bounded poll: true once the phase with the given parity has completed
__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_polls(uint64_t* bar, unsigned parity, long long polls)
{
    for (long long k = 0; k < polls; ++k)
        if (mbar_test(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity)
{
    return mbar_wait_polls(bar, parity, kMbarSpinLimit);
}
// plain arrival (release at CTA scope): the phase completes once every expected
// thread has arrived
__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(a) : "memory");
}

}  // namespace lbmk
