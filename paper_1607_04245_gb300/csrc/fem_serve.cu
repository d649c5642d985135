// fem_serve.cu -- the per-request launch of the serving loop in native code: one call
// uploads a request's inputs (one pinned host block laid out like the leading part of its
// device block), runs its kernels, downloads its results and records its completion
// event, all on the request's stream; a second call tests many completion events at
// once. A host-side scheduler above the C ABI (arrival, admission by arena footprint,
// statistics) calls these two per request; fem_serve_run, at the end of this file, is the
// same scheduling as one native call over a whole stream.
#include "fem_internal.cuh"

using namespace fem;

extern "C" int64_t fem_serve_request_bytes(void) { return static_cast<int64_t>(sizeof(fem_serve_request)); }

extern "C" fem_status fem_serve_event_create(void **event) {
    if (!event) return fail(FEM_ERR_ARG, "event is NULL");
    cudaEvent_t e = nullptr;
    const cudaError_t err = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (err != cudaSuccess) return fail(FEM_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(err));
    *event = e;
    return FEM_OK;
}

extern "C" void fem_serve_event_destroy(void *event) {
    if (event) cudaEventDestroy(static_cast<cudaEvent_t>(event));
}

extern "C" fem_status fem_serve_events_query(void *const *events, int n, int *done) {
    if (n < 0 || (n > 0 && (!events || !done))) return fail(FEM_ERR_ARG, "bad event list");
    for (int i = 0; i < n; ++i) {
        const cudaError_t e = cudaEventQuery(static_cast<cudaEvent_t>(events[i]));
        if (e == cudaSuccess) {
            done[i] = 1;
        } else if (e == cudaErrorNotReady) {
            done[i] = 0;
        } else {
            return fail(FEM_ERR_CUDA, "cudaEventQuery: %s", cudaGetErrorString(e));
        }
    }
    return FEM_OK;
}

// Bytes of every array a request uses (0: slot unused), from its sizes and precision.
static fem_status slot_bytes(const fem_serve_request *r, int64_t (&bytes)[FEM_SERVE_SLOTS]) {
    for (auto &b : bytes) b = 0;
    if (r->kind == 2) return FEM_OK;  // the self-test uses no arrays
    if (r->dim != 2 && r->dim != 3) return fail(FEM_ERR_ARG, "dim = %d, must be 2 or 3", r->dim);
    if (r->n_q < 1 || r->n_q > FEM_MAX_QPTS) return fail(FEM_ERR_ARG, "n_q = %d", r->n_q);
    if (r->n_cells < 0 || r->n_cells > INT32_MAX || r->n_verts < 0 || r->n_verts > INT32_MAX)
        return fail(FEM_ERR_ARG, "n_cells or n_verts out of range");
    int64_t s;
    switch (r->prec) {
        case FEM_FP64: case FEM_FP64_DF: s = 8; break;
        case FEM_FP32_MIXED: case FEM_FP32: s = 4; break;
        default: return fail(FEM_ERR_ARG, "unknown precision %d", r->prec);
    }
    const int64_t d = r->dim, C = r->n_cells, V = r->n_verts, nq = r->n_q, nc = r->physics == 0 ? 1 : d;
    bytes[FEM_SERVE_COORDS] = d * V * 8;
    bytes[FEM_SERVE_CONN] = (d + 1) * C * 4;
    bytes[FEM_SERVE_U] = nc * V * s;
    bytes[FEM_SERVE_K] = nq * C * s;
    if (r->physics == 1) bytes[FEM_SERVE_MU] = nq * C * s;
    if (r->kind == 0) {
        bytes[FEM_SERVE_OUT] = (d + 1) * nc * C * s;
    } else {
        bytes[FEM_SERVE_ADJ] = (d + 1) * C * s;
        bytes[FEM_SERVE_OUT] = nq * C * s;
        bytes[FEM_SERVE_DU] = V * s;
        bytes[FEM_SERVE_SCRATCH] = (d + 1) * C * s;
        bytes[FEM_SERVE_NODE_PTR] = (V + 1) * 4;
        bytes[FEM_SERVE_NODE_IDX] = (d + 1) * C * 4;
        bytes[FEM_SERVE_WORK] = fem_node2cell_work_size(V) * 4;
    }
    return FEM_OK;
}

extern "C" fem_status fem_serve_launch(const fem_serve_request *r, void *block, void *event, fem_stream stream) {
    if (!r || !block || !event) return fail(FEM_ERR_ARG, "a NULL argument");
    if (r->kind < 0 || r->kind > 2) return fail(FEM_ERR_ARG, "kind = %d", r->kind);
    if (r->physics != 0 && r->physics != 1) return fail(FEM_ERR_ARG, "physics = %d", r->physics);
    if (r->kind == 1 && r->physics != 0) return fail(FEM_ERR_UNSUPPORTED, "adjoint requests are Laplacian only");
    if (r->in_bytes < 0 || r->out_bytes[0] < 0 || r->out_bytes[1] < 0) return fail(FEM_ERR_ARG, "negative size");
    // the descriptor against its block: nothing below may touch memory outside it
    int64_t need[FEM_SERVE_SLOTS];
    fem_status vs = slot_bytes(r, need);
    if (vs != FEM_OK) return vs;
    if (r->block_bytes <= 0 || r->in_bytes > r->block_bytes) return fail(FEM_ERR_ARG, "in_bytes exceeds block_bytes");
    for (int k = 0; k < FEM_SERVE_SLOTS; ++k) {
        if (need[k] == 0) continue;
        if (r->offset[k] < 0 || r->offset[k] > r->block_bytes - need[k])
            return fail(FEM_ERR_ARG, "array %d (%lld bytes at offset %lld) outside the %lld-byte block", k,
                        static_cast<long long>(need[k]), static_cast<long long>(r->offset[k]),
                        static_cast<long long>(r->block_bytes));
    }
    if (r->out_bytes[0] > need[FEM_SERVE_OUT] || r->out_bytes[1] > need[FEM_SERVE_DU])
        return fail(FEM_ERR_ARG, "out_bytes larger than the arrays they copy");
    unsigned *status_dev = nullptr;  // the device's address of host_status
    if (r->host_status) {
        // the kernels write this word: it must be host memory the device can reach
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, r->host_status) != cudaSuccess || pa.type != cudaMemoryTypeHost ||
            !pa.devicePointer || (reinterpret_cast<uintptr_t>(r->host_status) & 3u)) {
            cudaGetLastError();
            return fail(FEM_ERR_ARG, "host_status must be a 4-byte aligned word of page-locked, device-mapped "
                                     "host memory");
        }
        status_dev = static_cast<unsigned *>(pa.devicePointer);
    }
    char *b = static_cast<char *>(block);
    auto at = [&](int slot) { return static_cast<void *>(b + r->offset[slot]); };
    const fem_precision prec = static_cast<fem_precision>(r->prec);
    cudaError_t e = cudaSuccess;
    if (r->in_bytes > 0) {
        if (!r->host_in) return fail(FEM_ERR_ARG, "host_in is NULL");
        e = cudaMemcpyAsync(b, r->host_in, size_t(r->in_bytes), cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return fail(FEM_ERR_CUDA, "fem_serve_launch upload: %s", cudaGetErrorString(e));
    }
    const double *coords = static_cast<const double *>(at(FEM_SERVE_COORDS));
    const int32_t *conn = static_cast<const int32_t *>(at(FEM_SERVE_CONN));
    // the request's own error word (mapped host memory, zeroed by the caller): every kernel
    // below reports into it
    struct Redirect {  // restores the device-wide word however this function returns
        explicit Redirect(unsigned *w) { set_error_word_override(w); }
        ~Redirect() { set_error_word_override(nullptr); }
    } redirect(status_dev);
    fem_status st = FEM_OK;
    if (r->kind == 2) {
        st = fem_selftest_wait(1000 * 1000, stream);  // a 1 ms wait that nothing completes
    } else if (r->kind == 0) {
        if (r->physics == 0)
            st = fem_integrate_laplacian(r->dim, r->n_cells, r->n_verts, coords, conn, at(FEM_SERVE_U),
                                         at(FEM_SERVE_K), r->n_q, r->qpts, r->qw, at(FEM_SERVE_OUT), prec, stream);
        else
            st = fem_integrate_elasticity(r->dim, r->n_cells, r->n_verts, coords, conn, at(FEM_SERVE_U),
                                          at(FEM_SERVE_K), at(FEM_SERVE_MU), r->n_q, r->qpts, r->qw,
                                          at(FEM_SERVE_OUT), prec, stream);
    } else {
        int32_t *ptr = static_cast<int32_t *>(at(FEM_SERVE_NODE_PTR));
        int32_t *idx = static_cast<int32_t *>(at(FEM_SERVE_NODE_IDX));
        st = fem_build_node2cell(r->dim, r->n_cells, r->n_verts, conn, ptr, idx,
                                 static_cast<int32_t *>(at(FEM_SERVE_WORK)), stream);
        if (st == FEM_OK)
            st = fem_adjoint_laplacian(r->dim, r->n_cells, r->n_verts, coords, conn, at(FEM_SERVE_U), at(FEM_SERVE_K),
                                       r->n_q, r->qpts, r->qw, at(FEM_SERVE_ADJ), at(FEM_SERVE_OUT),
                                       at(FEM_SERVE_DU), ptr, idx, at(FEM_SERVE_SCRATCH), prec, stream);
    }
    if (st != FEM_OK) return st;
    // results: out (residual) or dK (adjoint) from slot OUT, du (adjoint) from slot DU
    const int src[2] = {FEM_SERVE_OUT, FEM_SERVE_DU};
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        if (r->out_bytes[k] == 0) continue;
        if (!r->host_out[k]) return fail(FEM_ERR_ARG, "host_out[%d] is NULL", k);
        e = cudaMemcpyAsync(r->host_out[k], at(src[k]), size_t(r->out_bytes[k]), cudaMemcpyDeviceToHost, stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(static_cast<cudaEvent_t>(event), stream);
    if (e != cudaSuccess) return fail(FEM_ERR_CUDA, "fem_serve_launch: %s", cudaGetErrorString(e));
    return FEM_OK;
}

// ------------------------------------------------------------------ the whole loop in native code
//
// fem_serve_run runs a stream of requests the way the host scheduler of serving.py does --
// a FIFO of arrived requests, admission as soon as a slot (a stream and its completion
// event) is free and the arena holds the request's footprint, backfill past a head that
// does not fit, completion by event -- without returning to the caller per request: the
// per-request host work is the launch call itself plus a few container operations.

#include <algorithm>
#include <chrono>
#include <deque>
#include <thread>
#include <vector>

namespace {

struct ServeRun {
    int n_slots;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    fem_arena *arena = nullptr;
    explicit ServeRun(int n) : n_slots(n), streams(n, nullptr), events(n, nullptr) {}
    ~ServeRun() {
        for (int s = 0; s < n_slots; ++s) {
            if (streams[s]) cudaStreamSynchronize(streams[s]);  // nothing of ours stays in flight
            if (events[s]) cudaEventDestroy(events[s]);
            if (streams[s]) cudaStreamDestroy(streams[s]);
        }
        if (arena) fem_arena_destroy(arena);
    }
};

}  // namespace

extern "C" fem_status fem_serve_run(const fem_serve_request *reqs, const int64_t *footprint, const double *arrival,
                                    int n, void *pool, int64_t pool_bytes, int64_t alignment, int n_slots,
                                    int backfill, fem_serve_result *results) {
    if (n < 0 || n_slots < 1 || n_slots > FEM_SERVE_MAX_SLOTS)
        return fail(FEM_ERR_ARG, "n = %d, n_slots = %d (1..%d)", n, n_slots, FEM_SERVE_MAX_SLOTS);
    if (n == 0) return FEM_OK;
    if (!reqs || !footprint || !arrival || !results || !pool) return fail(FEM_ERR_ARG, "a NULL argument");
    if (pool_bytes <= 0) return fail(FEM_ERR_ARG, "pool_bytes must be positive");
    if (alignment < 256 || (alignment & (alignment - 1)) != 0)
        return fail(FEM_ERR_ARG, "alignment = %lld, must be a power of two >= 256", static_cast<long long>(alignment));
    if (reinterpret_cast<uintptr_t>(pool) % static_cast<uintptr_t>(alignment) != 0)
        return fail(FEM_ERR_ARG, "pool is not aligned to %lld bytes", static_cast<long long>(alignment));
    for (int i = 0; i < n; ++i)
        if (!(arrival[i] >= 0.0 && arrival[i] < 1e9) || footprint[i] < 0)
            return fail(FEM_ERR_ARG, "request %d: arrival %g or footprint %lld", i, arrival[i],
                        static_cast<long long>(footprint[i]));
    ServeRun run(n_slots);
    fem_status st = fem_arena_create(pool_bytes, alignment, &run.arena);
    if (st != FEM_OK) return st;
    for (int s = 0; s < n_slots; ++s) {
        cudaError_t e = cudaStreamCreateWithFlags(&run.streams[s], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&run.events[s], cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(FEM_ERR_CUDA, "fem_serve_run: %s", cudaGetErrorString(e));
    }
    const int64_t capacity = fem_arena_capacity(run.arena);
    auto rounded = [&](int64_t b) { return b == 0 ? alignment : (b + alignment - 1) / alignment * alignment; };
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return arrival[x] < arrival[y]; });
    for (int i = 0; i < n; ++i) results[i] = fem_serve_result{-1.0, -1.0, -1.0, -1, 0u};
    struct Slot {
        int req = -1;
        int64_t offset = 0;
        bool refused = false;  // its launch was refused: nothing but (maybe) its upload ran
    };
    std::vector<Slot> slots(n_slots);
    std::vector<int> free_slots;
    for (int s = n_slots - 1; s >= 0; --s) free_slots.push_back(s);
    std::deque<int> queue;
    const auto t0 = std::chrono::steady_clock::now();
    auto now_s = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
    int next = 0, finished = 0, inflight = 0;
    while (finished < n) {
        const double t = now_s();
        while (next < n && arrival[order[next]] <= t) {
            const int r = order[next++];
            results[r].t_arrive = arrival[r];
            if (rounded(footprint[r]) > capacity) {  // can never run: rejected on arrival
                results[r].t_done = now_s();
                results[r].status = FEM_SERVE_REJECTED;
                ++finished;
            } else {
                queue.push_back(r);
            }
        }
        bool progressed = false;
        if (!free_slots.empty() && !queue.empty()) {
            int64_t largest = fem_arena_largest_free(run.arena);
            for (size_t i = 0; i < queue.size() && !free_slots.empty();) {
                const int r = queue[i];
                int64_t off = 0;
                if (rounded(footprint[r]) > largest || fem_arena_alloc(run.arena, footprint[r], &off) != FEM_OK) {
                    if (!backfill) break;
                    ++i;
                    continue;
                }
                const int s = free_slots.back();
                free_slots.pop_back();
                if (reqs[r].host_status) *static_cast<volatile unsigned *>(reqs[r].host_status) = 0u;
                fem_serve_request rq = reqs[r];
                rq.block_bytes = footprint[r];
                results[r].t_admit = now_s();
                st = fem_serve_launch(&rq, static_cast<char *>(pool) + off, run.events[s], run.streams[s]);
                bool refused = false;
                if (st == FEM_ERR_CUDA) return st;  // the device or the runtime failed: stop
                if (st != FEM_OK) {
                    // a descriptor the launcher refused: the request fails, the stream goes on; its
                    // block stays held until whatever it enqueued has drained
                    refused = true;
                    const cudaError_t e = cudaEventRecord(run.events[s], run.streams[s]);
                    if (e != cudaSuccess) return fail(FEM_ERR_CUDA, "fem_serve_run: %s", cudaGetErrorString(e));
                }
                slots[s] = Slot{r, off, refused};
                queue.erase(queue.begin() + static_cast<std::ptrdiff_t>(i));
                ++inflight;
                progressed = true;
                largest = fem_arena_largest_free(run.arena);
            }
        }
        for (int s = 0; s < n_slots && inflight > 0; ++s) {
            if (slots[s].req < 0) continue;
            const cudaError_t q = cudaEventQuery(run.events[s]);
            if (q == cudaErrorNotReady) continue;
            const int r = slots[s].req;
            if (q != cudaSuccess)
                return fail(FEM_ERR_CUDA, "fem_serve_run: request %d: %s", r, cudaGetErrorString(q));
            results[r].t_done = now_s();
            if (slots[s].refused) {
                results[r].status = FEM_SERVE_REFUSED;
            } else {
                const unsigned bits =
                    reqs[r].host_status ? *static_cast<volatile unsigned *>(reqs[r].host_status) : 0u;
                results[r].bits = bits;
                results[r].status = bits ? FEM_SERVE_FAILED : FEM_SERVE_DONE;
            }
            fem_arena_free(run.arena, slots[s].offset);
            slots[s] = Slot{};
            free_slots.push_back(s);
            --inflight;
            ++finished;
            progressed = true;
        }
        if (!progressed && inflight == 0 && queue.empty() && next < n) {
            // idle until the next arrival: sleeps of at most 1 ms, the last 0.2 ms spun
            const double wait = arrival[order[next]] - now_s();
            if (wait > 2e-4) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait - 2e-4, 1e-3)));
        }
    }
    return FEM_OK;
}
