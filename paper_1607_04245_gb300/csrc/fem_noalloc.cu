// fem_noalloc.cu -- the Laplacian adjoint for callers that cannot allocate device memory.
//
// fem_adjoint_laplacian needs a caller-provided workspace of (dim+1) * n_cells values
// for the per-element part of dJ/du. Some callers have no such buffer to hand over and
// cannot obtain one: code that is given only the input and output pointers (a plugin
// or a callback inside a host framework that owns all device memory), or a loop that
// must not call cudaMalloc because of the device-wide synchronisation it implies. This
// file gives them fem_adjoint_laplacian_noalloc, which takes its workspace from a
// fixed-size array in the library's own device memory instead.
//
// The array is a file-scope static __device__ object: every GPU that loads the library
// holds FEM_NOALLOC_SCRATCH_BYTES of it until the process exits. In host code its name
// is only a host-side stand-in, so the device address is looked up with
// cudaGetSymbolAddress, once per device, with that device current, on the first call
// made on that device.
#include <cstdio>
#include <mutex>

#include "fem_internal.cuh"

static __device__ __align__(256) unsigned char g_noalloc_scratch[FEM_NOALLOC_SCRATCH_BYTES];

namespace fem {

static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[256] = {nullptr};

// Device address of g_noalloc_scratch on the current device (looked up once per device and
// kept for the life of the process: a device reset after the first call is not supported).
static fem_status noalloc_scratch(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(FEM_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 256) return fail(FEM_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(FEM_ERR_CUDA, "cudaGetSymbolAddress(g_noalloc_scratch) on device %d: %s", dev,
                        cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return FEM_OK;
}

}  // namespace fem

using namespace fem;

extern "C" fem_status fem_adjoint_laplacian_noalloc(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                                    const int32_t *conn, const void *u, const void *K, int n_q,
                                                    const double *qpts, const double *qw, const void *lambda,
                                                    void *dK, void *du, const int32_t *node_ptr,
                                                    const int32_t *node_idx, fem_precision prec, fem_stream stream) {
    if (dim != 2 && dim != 3) return fail(FEM_ERR_ARG, "dim = %d, must be 2 or 3", dim);
    if (n_cells < 0) return fail(FEM_ERR_ARG, "negative n_cells");
    if (prec != FEM_FP64 && prec != FEM_FP32_MIXED && prec != FEM_FP32 && prec != FEM_FP64_DF)
        return fail(FEM_ERR_ARG, "unknown precision %d", static_cast<int>(prec));
    const int64_t value_bytes = (prec == FEM_FP64 || prec == FEM_FP64_DF) ? 8 : 4;
    const int64_t need = int64_t(dim + 1) * n_cells * value_bytes;
    if (need > int64_t(FEM_NOALLOC_SCRATCH_BYTES))
        return fail(FEM_ERR_SHAPE,
                    "fem_adjoint_laplacian_noalloc: %lld cells need %lld bytes of workspace, more than the "
                    "library's fixed %lld-byte array; use fem_adjoint_laplacian with a caller-owned workspace",
                    static_cast<long long>(n_cells), static_cast<long long>(need),
                    static_cast<long long>(FEM_NOALLOC_SCRATCH_BYTES));
    void *scratch = nullptr;
    fem_status st = noalloc_scratch(&scratch);
    if (st != FEM_OK) return st;
    // Every workspace entry the gather reads is written by the element kernel earlier in
    // this same call, so nothing has to be cleared between calls -- unless a staged element
    // kernel gave up a bounded wait (FEM_ERR_TIMEOUT from fem_device_error): it then skips
    // that tile's writes, and du mixes in the previous call's values; the header says so.
    return fem_adjoint_laplacian(dim, n_cells, n_verts, coords, conn, u, K, n_q, qpts, qw, lambda, dK, du, node_ptr,
                                 node_idx, scratch, prec, stream);
}
