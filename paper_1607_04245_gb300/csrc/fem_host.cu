// fem_host.cu -- the Laplacian residual for data that lives in host memory. The vertex
// arrays are uploaded once (every cell gathers from them). The cell-indexed arrays then
// take one of two routes:
//   * chunks >= 1: the cells are processed in chunks on two internal streams, so that the
//     upload of one chunk, the kernel of another and the download of a third overlap
//     (host <-> device copies run in both directions at once);
//   * chunks == 0: no copies; the kernel reads the connectivity and coefficient rows from
//     the page-locked host arrays and writes the element vectors back to host memory
//     across the host link, so the transfer in each direction runs for the whole kernel
//     instead of being cut into copy-engine transfers with a fill and a drain.
// The device buffers come from a caller-provided workspace; nothing is allocated.
#include <mutex>

#include "fem_internal.cuh"

namespace fem {

constexpr int kHostStreams = 2;

struct HostStreams {
    cudaStream_t s[kHostStreams] = {nullptr, nullptr};
    cudaEvent_t ready = nullptr, done[kHostStreams] = {nullptr, nullptr};
    bool ok = false;
};

// streams and events of the current device, created on first use and kept for the life
// of the process
static fem_status host_streams(HostStreams *&out) {
    static std::mutex mu;
    static HostStreams per_dev[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return fail(FEM_ERR_CUDA, "cudaGetDevice failed");
    std::lock_guard<std::mutex> lk(mu);
    HostStreams &h = per_dev[dev];
    if (!h.ok) {
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < kHostStreams && e == cudaSuccess; ++i) {
            e = cudaStreamCreateWithFlags(&h.s[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.done[i], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.ready, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(FEM_ERR_CUDA, "host-path streams: %s", cudaGetErrorString(e));
        h.ok = true;
    }
    out = &h;
    return FEM_OK;
}

static size_t a256(size_t n) { return (n + 255) & ~size_t(255); }

// the device address of page-locked, mapped host memory; false for anything else
static bool mapped_host_ptr(const void *h, void *&d) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return false;
    void *m = nullptr;
    if (cudaHostGetDevicePointer(&m, const_cast<void *>(h), 0) != cudaSuccess || !m) {
        cudaGetLastError();
        return false;
    }
    d = m;
    return true;
}

struct HostLayout {
    size_t coords, u, conn[kHostStreams], K[kHostStreams], out[kHostStreams], total;
    int64_t chunk;  // cells per chunk (multiple of 4)
};

static HostLayout host_layout(int dim, int64_t C, int64_t V, int n_q, size_t vs, int chunks) {
    HostLayout L;
    const int nb = dim + 1;
    if (chunks == 0) {  // vertex arrays only
        L.chunk = 0;
        L.coords = 0;
        L.u = a256(size_t(dim) * V * sizeof(double));
        L.total = L.u + a256(size_t(V) * vs);
        for (int i = 0; i < kHostStreams; ++i) L.conn[i] = L.K[i] = L.out[i] = 0;
        return L;
    }
    int64_t per = (C + chunks - 1) / chunks;
    per = (per + 3) / 4 * 4;
    L.chunk = per < 4 ? 4 : per;
    size_t off = 0;
    L.coords = off, off += a256(size_t(dim) * V * sizeof(double));
    L.u = off, off += a256(size_t(V) * vs);
    for (int i = 0; i < kHostStreams; ++i) {
        L.conn[i] = off, off += a256(size_t(nb) * L.chunk * 4);
        L.K[i] = off, off += a256(size_t(n_q) * L.chunk * vs);
        L.out[i] = off, off += a256(size_t(nb) * L.chunk * vs);
    }
    L.total = off;
    return L;
}

fem_status integrate_laplacian_plain(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                     const int32_t *conn, const void *u, const void *K, int n_q, const double *qpts,
                                     const double *qw, void *elem_out, fem_precision prec, cudaStream_t stream);

}  // namespace fem

using namespace fem;

extern "C" int64_t fem_host_work_bytes(int dim, int64_t n_cells, int64_t n_verts, int n_q, fem_precision prec,
                                       int chunks) {
    if ((dim != 2 && dim != 3) || n_cells < 0 || n_verts < 0 || n_q < 1 || chunks < 0) return -1;
    return static_cast<int64_t>(host_layout(dim, n_cells, n_verts, n_q, prec == FEM_FP64 ? 8 : 4, chunks).total);
}

extern "C" fem_status fem_integrate_laplacian_host(int dim, int64_t n_cells, int64_t n_verts, const double *coords_h,
                                                   const int32_t *conn_h, const void *u_h, const void *K_h, int n_q,
                                                   const double *qpts, const double *qw, void *out_h, void *work,
                                                   int64_t work_bytes, int chunks, fem_precision prec,
                                                   fem_stream stream) {
    fem_status st = check_common(dim, n_cells, n_verts, coords_h, conn_h);
    if (st != FEM_OK) return st;
    if (prec != FEM_FP64 && prec != FEM_FP32_MIXED && prec != FEM_FP32)
        return fail(FEM_ERR_ARG, "unknown precision %d", static_cast<int>(prec));
    if (chunks < 0) return fail(FEM_ERR_ARG, "chunks must be >= 0");
    if (n_q < 1 || n_q > FEM_MAX_QPTS) return fail(FEM_ERR_SHAPE, "n_q = %d outside [1, %d]", n_q, FEM_MAX_QPTS);
    if (n_cells == 0) return FEM_OK;
    if (!u_h || !K_h || !out_h || !work) return fail(FEM_ERR_ARG, "a NULL array argument");
    const size_t vs = prec == FEM_FP64 ? 8 : 4;
    const HostLayout L = host_layout(dim, n_cells, n_verts, n_q, vs, chunks);
    if (work_bytes < static_cast<int64_t>(L.total))
        return fail(FEM_ERR_OOM, "fem_integrate_laplacian_host: workspace of %lld bytes, %lld needed",
                    static_cast<long long>(work_bytes), static_cast<long long>(L.total));
    if (reinterpret_cast<uintptr_t>(work) & 255u) return fail(FEM_ERR_ARG, "work must be 256-byte aligned");
    char *w = static_cast<char *>(work);
    const int nb = dim + 1;
    cudaError_t e = cudaSuccess;
    if (chunks == 0) {
        // device addresses of the page-locked host arrays; pageable memory (which a kernel
        // must not be handed) is refused here
        void *conn_m = nullptr, *K_m = nullptr, *out_m = nullptr;
        if (!mapped_host_ptr(conn_h, conn_m) || !mapped_host_ptr(K_h, K_m) || !mapped_host_ptr(out_h, out_m))
            return fail(FEM_ERR_ARG, "fem_integrate_laplacian_host (chunks = 0): conn_h, K_h and out_h must be "
                        "page-locked, device-mapped host memory");
        double *coords_d = reinterpret_cast<double *>(w + L.coords);
        void *u_d = w + L.u;
        e = cudaMemcpyAsync(coords_d, coords_h, size_t(dim) * n_verts * sizeof(double), cudaMemcpyHostToDevice,
                            stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(u_d, u_h, size_t(n_verts) * vs, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return fail(FEM_ERR_CUDA, "fem_integrate_laplacian_host: %s", cudaGetErrorString(e));
        return integrate_laplacian_plain(dim, n_cells, n_verts, coords_d, static_cast<const int32_t *>(conn_m), u_d,
                                         K_m, n_q, qpts, qw, out_m, prec, stream);
    }
    HostStreams *hs = nullptr;
    if ((st = host_streams(hs)) != FEM_OK) return st;
    // vertex arrays, once, on the caller's stream; the chunk streams wait for them
    double *coords_d = reinterpret_cast<double *>(w + L.coords);
    void *u_d = w + L.u;
    e = cudaMemcpyAsync(coords_d, coords_h, size_t(dim) * n_verts * sizeof(double), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(u_d, u_h, size_t(n_verts) * vs, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaEventRecord(hs->ready, stream);
    for (int i = 0; i < kHostStreams && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(hs->s[i], hs->ready, 0);
    if (e != cudaSuccess) return fail(FEM_ERR_CUDA, "fem_integrate_laplacian_host: %s", cudaGetErrorString(e));
    const int64_t nchunks = (n_cells + L.chunk - 1) / L.chunk;
    for (int64_t k = 0; k < nchunks; ++k) {
        const int i = static_cast<int>(k % kHostStreams);
        cudaStream_t s = hs->s[i];
        const int64_t c0 = k * L.chunk;
        const int64_t cc = n_cells - c0 < L.chunk ? n_cells - c0 : L.chunk;
        int32_t *conn_d = reinterpret_cast<int32_t *>(w + L.conn[i]);
        void *K_d = w + L.K[i], *out_d = w + L.out[i];
        // rows of the chunk: [nb][cc] conn, [n_q][cc] K (host row pitch n_cells)
        e = cudaMemcpy2DAsync(conn_d, cc * 4, conn_h + c0, n_cells * 4, cc * 4, nb, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(K_d, cc * vs, static_cast<const char *>(K_h) + c0 * vs, n_cells * vs, cc * vs, n_q,
                                  cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return fail(FEM_ERR_CUDA, "fem_integrate_laplacian_host: %s", cudaGetErrorString(e));
        st = fem_integrate_laplacian(dim, cc, n_verts, coords_d, conn_d, u_d, K_d, n_q, qpts, qw, out_d, prec, s);
        if (st != FEM_OK) return st;
        e = cudaMemcpy2DAsync(static_cast<char *>(out_h) + c0 * vs, n_cells * vs, out_d, cc * vs, cc * vs, nb,
                              cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return fail(FEM_ERR_CUDA, "fem_integrate_laplacian_host: %s", cudaGetErrorString(e));
    }
    // the caller's stream completes when every chunk has been downloaded
    for (int i = 0; i < kHostStreams && e == cudaSuccess; ++i) {
        e = cudaEventRecord(hs->done[i], hs->s[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, hs->done[i], 0);
    }
    if (e != cudaSuccess) return fail(FEM_ERR_CUDA, "fem_integrate_laplacian_host: %s", cudaGetErrorString(e));
    return FEM_OK;
}
