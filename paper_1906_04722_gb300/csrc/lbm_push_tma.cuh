// lbm_push_tma.cuh -- what the push-form step kernels share: bounded mbarrier
// waits, tensor-memory-accelerator box loads (with and without an L2 eviction
// policy) and prefetches, and the conversion of pull bounce bits into push
// bounce bits.
#pragma once

#include <cuda.h>

#include <cstdint>

namespace lbmk {

constexpr long long PUSH_WAIT_NS = 2000000000LL;  // 2 s
constexpr uint32_t PUSH_BOUNCE_BITS = 0x7fffeu;   // bits 1..18

__device__ __forceinline__ uint32_t p_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void p_mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(p_smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void p_mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(p_smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void p_mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(p_smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool p_mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(p_smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ unsigned long long p_global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of the given parity, for at most PUSH_WAIT_NS.
__device__ __forceinline__ bool p_mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (p_mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = p_global_ns();
    while (true) {
        for (int i = 0; i < 64; ++i)
            if (p_mbar_try_wait(bar, parity)) return true;
        if ((long long)(p_global_ns() - t0) > PUSH_WAIT_NS) return false;
    }
}
__device__ __forceinline__ void p_tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                              uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(p_smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(p_smem_u32(bar))
        : "memory");
}

// The same load with an L2 eviction policy (from createpolicy) attached.
__device__ __forceinline__ void p_tma_load_4d_hint(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                                   uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, "
        "{%2, %3, %4, %5}], [%6], %7;\n" ::"r"(p_smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(p_smem_u32(bar)), "l"(policy)
        : "memory");
}
__device__ __forceinline__ uint64_t p_policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}

// A hint: the box at these coordinates into L2, nothing into shared memory and
// no completion to wait for.
__device__ __forceinline__ void p_tma_prefetch_4d(const CUtensorMap* map, int c0, int c1, int c2, int c3) {
    asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];\n" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(c0), "r"(c1), "r"(c2), "r"(c3)
                 : "memory");
}

// Swaps the bits of each opposite pair: pull bounce bits (x - e_k not fluid)
// become push bounce bits (x + e_k not fluid).
__device__ __forceinline__ uint32_t p_swap_pairs(uint32_t m) {
    return ((m & 0x2aaaau) << 1) | ((m & 0x55554u) >> 1);
}

// Tile mode, three dimensions, the same completion as the 4-D load.
__device__ __forceinline__ void p_tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                              uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(p_smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(p_smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void p_tma_load_3d_hint(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                                   uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, "
        "{%2, %3, %4}], [%5], %6;\n" ::"r"(p_smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(p_smem_u32(bar)), "l"(policy)
        : "memory");
}

}  // namespace lbmk
