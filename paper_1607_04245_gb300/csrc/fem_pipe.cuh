// fem_pipe.cuh -- asynchronous staging of cell-indexed rows into shared memory.
//
// The staged kernels are persistent: each CTA walks a strided sequence of tiles of
// consecutive cells. One elected thread copies the tile's rows of every cell-indexed
// input (connectivity, coefficients, adjoint weights) from global into a ring of
// shared-memory stages with the bulk-copy engine (cp.async.bulk, completion counted in
// bytes on an mbarrier), several tiles ahead of the consumers. The consumer threads
// then read their cells from shared memory, so no thread holds a DRAM round trip on
// its own dependence chain except the vertex gathers.
//
// Every wait is bounded (a %globaltimer budget); a wait that runs out records
// FEM_DEVERR_TIMEOUT in the library's device error word, waits (again bounded) for the
// stage copies it issued, and returns without touching the outputs of that tile.
#pragma once

#include <stdint.h>

#include "fem_internal.cuh"

namespace fem {

// Device error word: bits set by kernels that gave up a bounded wait. It lives in
// fem_core.cu; kernels get its device address (device_error_word()) as an argument.
// fem_device_error() reads and clears it.
enum : unsigned { FEM_DEVERR_TIMEOUT = 1u };
unsigned *device_error_word();

// budget of one bounded wait (nanoseconds of %globaltimer)
constexpr uint64_t kWaitBudgetNs = 500ull * 1000ull * 1000ull;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// make the barrier initialisation visible to the bulk-copy (async) proxy
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// plain arrival (no transaction bytes)
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
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

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase with the given parity to complete; false when the budget ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t budget_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_timer_ns() - t0 > budget_ns) return false;
    return true;
}

// L2 policy for data read exactly once: evict first, so the gathered vertex arrays stay.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from global to
// this CTA's shared memory; completion is counted on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                              uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ void record_device_error(unsigned *err, unsigned bits) { atomicOr(err, bits); }

}  // namespace fem
