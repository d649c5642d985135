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
#include <string.h>

#include "fem_internal.cuh"

namespace fem {

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

// ------------------------------------------------------------------ the staged chunk loop
//
// Persistent CTAs walk the chunks of kTile consecutive cells round-robin (chunk
// blockIdx.x, blockIdx.x + gridDim.x, ...), so that at any time the CTAs of the device
// work on one contiguous front of the cell arrays (DRAM pages and the L2-resident vertices
// of neighbouring chunks are shared). The CTA is warp-specialised: one producer warp
// brings each chunk's cell-indexed rows into a ring of shared-memory stages with the
// bulk-copy engine ("full" barriers count the bytes), and kConsumerWarps consumer warps
// compute. Consumer warps release a stage on its "empty" barrier as soon as they are done
// with it; there is no CTA-wide barrier per chunk, so the warps drift apart and one warp's
// vertex gathers overlap other warps' arithmetic. Within a chunk each consumer thread owns
// kCPT consecutive cells. Tuning (measured on the 1,572,864-tet Laplacian workload): 4
// cells per consumer thread, 8 consumer warps, 2 CTAs per SM and a 64 KB stage budget.
#ifndef FEM_STAGED_MIN_CTAS
#define FEM_STAGED_MIN_CTAS 2
#endif
#ifndef FEM_STAGED_BUDGET_KB
#define FEM_STAGED_BUDGET_KB 64
#endif
#ifndef FEM_STAGED_CPT
#define FEM_STAGED_CPT 4
#endif
#ifndef FEM_STAGED_CWARPS
#define FEM_STAGED_CWARPS 8
#endif
constexpr int kCPT = FEM_STAGED_CPT;
constexpr int kConsumerWarps = FEM_STAGED_CWARPS;
constexpr int kTile = kCPT * 32 * kConsumerWarps;
constexpr int kMaxStages = 4;
constexpr int kStagedThreads = 32 * kConsumerWarps + 32;  // consumers + one producer warp
static_assert(kCPT == 2 || kCPT == 4, "two or four cells per thread");
// shared-memory budget of the ring (per CTA) and the largest stage pair a CTA may hold
constexpr uint32_t kStageBudget = uint32_t(FEM_STAGED_BUDGET_KB) << 10;
constexpr uint32_t kStageMax = 200u << 10;

// Stages in the ring for stages of `stage_bytes` each (at least two: copy ahead of use).
inline int ring_stages(uint32_t stage_bytes) {
    const uint32_t n = kStageBudget / stage_bytes;
    return static_cast<int>(n < 2u ? 2u : (n > uint32_t(kMaxStages) ? uint32_t(kMaxStages) : n));
}

// CPT consecutive values of a cell-indexed row in shared memory (one vector load)
template <int CPT, class T>
__device__ __forceinline__ void lds_row(const T *p, T (&v)[CPT]) {
    static_assert(CPT == 2 || CPT == 4, "two or four cells per thread");
    if constexpr (sizeof(T) * CPT == 8) {
        const uint2 t = *reinterpret_cast<const uint2 *>(p);
        memcpy(&v[0], &t.x, 4), memcpy(&v[1], &t.y, 4);
    } else if constexpr (sizeof(T) * CPT == 16) {
        const uint4 t = *reinterpret_cast<const uint4 *>(p);
        memcpy(&v[0], &t, 16);
    } else {
        const uint4 t0 = reinterpret_cast<const uint4 *>(p)[0], t1 = reinterpret_cast<const uint4 *>(p)[1];
        memcpy(&v[0], &t0, 16), memcpy(&v[2], &t1, 16);
    }
}

// The chunk loop of a staged kernel launched with kStagedThreads threads and
// `stages` * stage-size bytes of dynamic shared memory. The producer lane calls
// issue(s, c0, n, bar) to start the bulk copies of the chunk of n cells at cell c0 into
// stage s (announcing their bytes on bar with mbar_arrive_expect_tx); every consumer
// thread whose cells j0 .. j0 + kCPT - 1 lie in the chunk calls work(s, c0, j0). The cell
// count C must be a multiple of kCPT, so that a thread's cells are all present or all
// absent. A wait that runs out sets FEM_DEVERR_TIMEOUT in *err; the producer drains its
// copies in flight before it leaves.
template <class Issue, class Work>
__device__ __forceinline__ void staged_chunks(int64_t C, int stages, unsigned *err, const Issue &issue,
                                              const Work &work) {
    __shared__ uint64_t full[kMaxStages], empty[kMaxStages];
    __shared__ volatile int s_abort;
    const int64_t ntiles = (C + kTile - 1) / kTile;
    // this CTA's chunks: tiles blockIdx.x + i * gridDim.x, i < nchunks
    const int64_t nchunks = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    auto chunk_start = [&](int64_t i) { return (blockIdx.x + i * gridDim.x) * int64_t(kTile); };
    auto chunk_cells = [&](int64_t i) {
        const int64_t c0 = chunk_start(i);
        return static_cast<uint32_t>(C - c0 < int64_t(kTile) ? C - c0 : int64_t(kTile));
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) mbar_init(&full[s], 1), mbar_init(&empty[s], kConsumerWarps);
        fence_barrier_init();
        s_abort = 0;
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == kConsumerWarps) {
        // ---------------- producer warp (one elected lane)
        if (lane != 0) return;
        int64_t issued = 0;
        for (int64_t i = 0; i < nchunks; ++i, ++issued) {
            const int s = static_cast<int>(i % stages);
            if (i >= stages) {
                // wait until every consumer warp has released the chunk i - stages
                const uint32_t par = static_cast<uint32_t>(((i / stages) - 1) & 1);
                if (s_abort || !mbar_wait_bounded(&empty[s], par, kWaitBudgetNs)) {
                    s_abort = 1;
                    break;
                }
            }
            issue(s, chunk_start(i), chunk_cells(i), &full[s]);
        }
        // drain: the last copies issued into each stage have landed before this warp leaves
        for (int64_t k = issued - stages < 0 ? 0 : issued - stages; k < issued; ++k)
            mbar_wait_bounded(&full[k % stages], static_cast<uint32_t>((k / stages) & 1), kWaitBudgetNs);
        if (s_abort) record_device_error(err, FEM_DEVERR_TIMEOUT);
        return;
    }

    // ---------------- consumer warps
    const int j0 = kCPT * threadIdx.x;
    for (int64_t i = 0; i < nchunks; ++i) {
        const int s = static_cast<int>(i % stages);
        if (s_abort || !mbar_wait_bounded(&full[s], static_cast<uint32_t>((i / stages) & 1), kWaitBudgetNs)) {
            s_abort = 1;
            record_device_error(err, FEM_DEVERR_TIMEOUT);
            return;
        }
        if (j0 < static_cast<int>(chunk_cells(i))) work(s, chunk_start(i), j0);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

}  // namespace fem
