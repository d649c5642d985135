// fem_serve.cu -- the per-request launch of the serving loop in native code: one call
// uploads a request's inputs (one pinned host block laid out like the leading part of its
// device block), runs its kernels, downloads its results and records its completion
// event, all on the request's stream; a second call tests many completion events at
// once. The host-side scheduler (arrival, admission by arena footprint, statistics) stays
// above the C ABI; what it calls per request is these two functions.
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

extern "C" fem_status fem_serve_launch(const fem_serve_request *r, void *block, void *event, fem_stream stream) {
    if (!r || !block || !event) return fail(FEM_ERR_ARG, "a NULL argument");
    if (r->kind != 0 && r->kind != 1) return fail(FEM_ERR_ARG, "kind = %d", r->kind);
    if (r->physics != 0 && r->physics != 1) return fail(FEM_ERR_ARG, "physics = %d", r->physics);
    if (r->kind == 1 && r->physics != 0) return fail(FEM_ERR_UNSUPPORTED, "adjoint requests are Laplacian only");
    if (r->in_bytes < 0 || r->out_bytes[0] < 0 || r->out_bytes[1] < 0) return fail(FEM_ERR_ARG, "negative size");
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
    fem_status st = FEM_OK;
    if (r->kind == 0) {
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
