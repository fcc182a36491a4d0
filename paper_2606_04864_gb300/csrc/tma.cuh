// TMA and mbarrier primitives shared by the local-solve kernels: bounded
// mbarrier waits, 2-D tensor copies into shared memory with optional L2
// eviction priorities, and the exit path after a wait runs out.
#pragma once

#include <cstdint>

#include <cuda.h>

#include "ams_internal.h"

namespace ams {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false when `budget` SM clock cycles pass without the phase
// of the given parity completing.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int64_t budget) {
    const long long t0 = clock64();
    do {
        if (mbar_try_wait(bar, parity)) return true;
    } while (clock64() - t0 < budget);
    return false;
}
// Budget of the exit drain (about a second): a copy in flight lands within
// microseconds, but the block must not leave while one may still write its
// shared memory.
constexpr int64_t kDrainCycles = int64_t(1) << 31;
// Exit path after a wait ran out: record the timeout, then wait for every
// copy this thread saw issued and not yet completed (slots with their bit
// in `pend`, at the parity they were issued with).
__device__ __forceinline__ void drain_copies(const uint64_t* bars, int nbuf, uint32_t pend, uint32_t phase) {
    for (int i = 0; i < nbuf; ++i)
        if ((pend >> i) & 1u) mbar_wait(smem_u32(bars + i), (phase >> i) & 1u, kDrainCycles);
}
__device__ __forceinline__ void timeout_drain(const uint64_t* bars, int nbuf, uint32_t pend, uint32_t phase,
                                              int32_t* err, SolveState* st, bool leader) {
    if (leader) {
        if (err != nullptr) atomicExch(err, (int)AMS_ERR_DEVICE_TIMEOUT);
        if (st != nullptr) st->done = 1;
    }
    drain_copies(bars, nbuf, pend, phase);
}
// Shared-memory mbarrier slots of a ring of nbuf copies: one per slot plus
// the probe barrier that nothing ever completes (timeout_probe), rounded up
// to an even count so that what follows stays 16-byte aligned.
__host__ __device__ __forceinline__ int ring_bar_slots(int nbuf) { return (nbuf + 2) & ~1; }
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
        ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// The same copy with an L2 eviction-priority hint (a createpolicy value).
__device__ __forceinline__ void tma_load_2d_hint(uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y,
                                                 uint32_t bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;\n"
        ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar), "l"(pol)
        : "memory");
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_normal() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}

// 1024-byte aligned start of the dynamic shared memory (the 128-byte swizzle
// pattern repeats every 1024 bytes).  Derived by pointer arithmetic, not an
// integer round trip, so that the compiler still sees a shared-memory
// pointer and emits shared-memory loads rather than generic ones.
__device__ __forceinline__ unsigned char* smem_align1024(unsigned char* p) {
    return p + ((1024u - (smem_u32(p) & 1023u)) & 1023u);
}

}  // namespace ams
