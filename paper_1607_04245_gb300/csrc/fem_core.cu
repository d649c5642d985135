// fem_core.cu -- status handling, argument checks, quadrature loading, launch sizing,
// and the ALU-rate probes used for the rooflines of the float64 kernels.
#include <atomic>
#include <map>
#include <tuple>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <utility>

#include "fem_cell.cuh"
#include "fem_pipe.cuh"

// Device error word of the staged kernels (see fem_pipe.cuh); one per device.
static __device__ unsigned g_fem_device_error = 0u;

namespace fem {

static thread_local char g_last_error[512] = "";
static std::atomic<float> g_mixed_tau{0.05f};

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

fem_status fail(fem_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return st;
}

fem_status check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(FEM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return FEM_OK;
}

fem_status load_quadrature(int dim, int n_q, const double *qpts, const double *qw, QuadW &out) {
    if (n_q < 1 || n_q > FEM_MAX_QPTS) return fail(FEM_ERR_SHAPE, "n_q = %d outside [1, %d]", n_q, FEM_MAX_QPTS);
    if (!qw) return fail(FEM_ERR_ARG, "qw is NULL");
    for (int q = 0; q < n_q; ++q) {
        if (!std::isfinite(qw[q])) return fail(FEM_ERR_ARG, "qw[%d] is not finite", q);
        out.wd[q] = qw[q];
        out.wf[q] = static_cast<float>(qw[q]);
    }
    for (int q = n_q; q < FEM_MAX_QPTS; ++q) out.wd[q] = 0.0, out.wf[q] = 0.0f;
    out.nq = n_q;
    if (qpts) {
        // the reference simplex: xi_k >= 0, sum_k xi_k <= 1 (small slack for rounding)
        for (int q = 0; q < n_q; ++q) {
            double s = 0.0;
            for (int k = 0; k < dim; ++k) {
                double x = qpts[q * dim + k];
                if (!(x >= -1e-12)) return fail(FEM_ERR_ARG, "qpts[%d] lies outside the reference simplex", q);
                s += x;
            }
            if (!(s <= 1.0 + 1e-12)) return fail(FEM_ERR_ARG, "qpts[%d] lies outside the reference simplex", q);
        }
    }
    return FEM_OK;
}

fem_status check_common(int dim, int64_t n_cells, int64_t n_verts, const double *coords, const int32_t *conn) {
    if (dim != 2 && dim != 3) return fail(FEM_ERR_ARG, "dim = %d, must be 2 or 3", dim);
    if (n_cells < 0 || n_verts < 0) return fail(FEM_ERR_ARG, "negative size");
    if (n_cells > 0 && n_verts < 1) return fail(FEM_ERR_SHAPE, "cells without vertices");
    if ((dim + 1) * n_cells >= (int64_t(1) << 31) || n_verts >= (int64_t(1) << 31))
        return fail(FEM_ERR_SHAPE, "mesh too large for int32 indexing");
    if (n_cells > 0 && (!coords || !conn)) return fail(FEM_ERR_ARG, "coords or conn is NULL");
    return FEM_OK;
}

float mixed_tau() { return g_mixed_tau.load(std::memory_order_relaxed); }

static thread_local unsigned *t_error_word_override = nullptr;

void set_error_word_override(unsigned *w) { t_error_word_override = w; }

// Device address of g_fem_device_error on the current device, looked up once per device
// (host code cannot use the symbol itself as a device pointer), unless the calling thread
// has redirected its launches to another word (set_error_word_override).
static unsigned *device_error_word_global();

unsigned *device_error_word() {
    return t_error_word_override ? t_error_word_override : device_error_word_global();
}

static unsigned *device_error_word_global() {
    static std::mutex mu;
    static unsigned *cached[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!cached[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_fem_device_error) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        cached[dev] = static_cast<unsigned *>(p);
    }
    return cached[dev];
}

int sm_count() {
    static std::atomic<int> cached[64] = {};  // per device; concurrent first calls store the same value
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int n = cached[dev].load(std::memory_order_relaxed);
    if (!n) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
        cached[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

// Resident CTAs per SM of a kernel launched with `block` threads and no dynamic shared
// memory (cached per device and kernel).
static int occupancy(const void *kernel, int block) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> occ_cache[64];  // per device, (kernel, block)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lk(mu);
    auto &cache = occ_cache[dev];
    const auto key = std::make_pair(kernel, block);
    auto it = cache.find(key);
    if (it == cache.end()) {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernel, block, 0) != cudaSuccess) {
            cudaGetLastError();  // clear the failed query only; the launch reports real errors
            o = 1;
        }
        it = cache.emplace(key, o < 1 ? 1 : o).first;
    }
    return it->second;
}

int resident_grid(const void *kernel, int block, int64_t n_threads) {
    const int64_t need = (n_threads + block - 1) / block;
    const int64_t cap = int64_t(occupancy(kernel, block)) * sm_count();
    const int64_t g = need < cap ? need : cap;
    return static_cast<int>(g < 1 ? 1 : g);
}

int grid_for(int64_t n_threads, int block, const void *kernel) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> occ_cache[64];  // per device, (kernel, block)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    int occ;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto &cache = occ_cache[dev];
        const auto key = std::make_pair(kernel, block);
        auto it = cache.find(key);
        if (it == cache.end()) {
            int o = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernel, block, 0) != cudaSuccess) {
                cudaGetLastError();  // clear the failed query only; the launch reports real errors
                o = 1;
            }
            it = cache.emplace(key, o < 1 ? 1 : o).first;
        }
        occ = it->second;
    }
    int64_t need = (n_threads + block - 1) / block;
    // grid-stride kernels: at most 8 full waves of resident CTAs
    int64_t cap = int64_t(8) * occ * sm_count();
    int64_t g = need < cap ? need : cap;
    return static_cast<int>(g < 1 ? 1 : g);
}

// Persistent grid of a staged kernel with `smem` bytes of dynamic shared memory: as many
// CTAs as fit on the device at once, at most one per tile. Raises the kernel's dynamic
// shared-memory limit on first use (per device and kernel).
fem_status staged_grid(const void *kernel, int block, size_t smem, int64_t n_tiles, int &grid) {
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, size_t>, int> occ_cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return fail(FEM_ERR_CUDA, "cudaGetDevice failed");
    int occ = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto &cache = occ_cache[dev];
        const auto key = std::make_tuple(kernel, block, smem);
        auto it = cache.find(key);
        if (it == cache.end()) {
            cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(smem));
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, block, smem);
            if (e != cudaSuccess || occ < 1) {
                cudaGetLastError();
                return fail(FEM_ERR_CUDA, "staged kernel does not fit: %zu bytes of shared memory (%s)", smem,
                            cudaGetErrorString(e));
            }
            it = cache.emplace(key, occ).first;
        }
        occ = it->second;
    }
    int64_t g = int64_t(occ) * sm_count();
    if (n_tiles < g) g = n_tiles;
    grid = static_cast<int>(g < 1 ? 1 : g);
    return FEM_OK;
}

// ------------------------------------------------------------------ probes

template <int KIND>
__global__ void __launch_bounds__(256) probe_kernel(int iters, void *out) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if constexpr (KIND == 0) {
        double a[8];
        const double b = 1.0 + 1e-9 * (threadIdx.x & 7), c = 1e-7;
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = 1.0 + i * 1e-3 + t * 1e-12;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < 8; ++i) s += a[i];
        static_cast<double *>(out)[t] = s;
    } else if constexpr (KIND == 1) {
        float a[8];
        const float b = 1.0f + 1e-6f * (threadIdx.x & 7), c = 1e-7f;
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = 1.0f + i * 1e-3f;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = fmaf(a[i], b, c);
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < 8; ++i) s += a[i];
        static_cast<float *>(out)[t] = s;
    } else if constexpr (KIND == 2) {
        float a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int lo = static_cast<int>(t);
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] += __double2float_rn(__hiloint2double(0x3ff00000 + i, lo + it));
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < 8; ++i) s += a[i];
        static_cast<float *>(out)[t] = s;
    } else {
        uint32_t a[8];
        const uint32_t b = 0x9e3779b9u ^ static_cast<uint32_t>(t), c = 0x7f4a7c15u;
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = static_cast<uint32_t>(t) * (i + 1);
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = ((a[i] ^ b) & 0x7fffffffu) + c;
        uint32_t s = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) s += a[i];
        static_cast<float *>(out)[t] = static_cast<float>(s);
    }
}

// Self-test of the bounded wait: one thread initialises an mbarrier that expects two
// arrivals, arrives once, and waits for a phase that can never complete.
__global__ void selftest_wait_kernel(uint64_t budget_ns, unsigned *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 2);
    fence_barrier_init();
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bar)) : "memory");
    if (!mbar_wait_bounded(&bar, 0, budget_ns)) record_device_error(err, FEM_DEVERR_TIMEOUT);
}

// The float64 kernels' quotient num / |den| (a Newton-Raphson reciprocal, fem_cell.cuh)
// beside the IEEE division num / fabs(den), element by element.
__global__ void selftest_quotient_kernel(int64_t n, const double *num, const double *den, double *q_lib,
                                         double *q_ieee) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        q_lib[i] = quot_abs(num[i], den[i]);
        q_ieee[i] = num[i] / fabs(den[i]);
    }
}

}  // namespace fem

using namespace fem;

extern "C" fem_status fem_selftest_quotient(int64_t n, const double *num, const double *den, double *q_lib,
                                            double *q_ieee, fem_stream stream) {
    if (n < 0) return fail(FEM_ERR_ARG, "negative n");
    if (n == 0) return FEM_OK;
    if (!num || !den || !q_lib || !q_ieee) return fail(FEM_ERR_ARG, "a NULL array");
    const int64_t blocks = (n + 255) / 256;
    selftest_quotient_kernel<<<static_cast<unsigned>(blocks < 4096 ? blocks : 4096), 256, 0, stream>>>(
        n, num, den, q_lib, q_ieee);
    return check_launch("fem_selftest_quotient");
}

extern "C" fem_status fem_device_error(fem_stream stream) {
    unsigned *w = device_error_word_global();
    if (!w) return fail(FEM_ERR_CUDA, "fem_device_error: device error word unavailable");
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail(FEM_ERR_CUDA, "fem_device_error: %s", cudaGetErrorString(e));
    unsigned v = 0;
    e = cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && v != 0u) {
        const unsigned zero = 0u;
        e = cudaMemcpy(w, &zero, sizeof(zero), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return fail(FEM_ERR_CUDA, "fem_device_error: %s", cudaGetErrorString(e));
    if (v & FEM_DEVERR_TIMEOUT)
        return fail(FEM_ERR_TIMEOUT, "a kernel gave up a bounded device-side wait%s",
                    (v & FEM_DEVERR_BADMESH) ? " (and a kernel met an invalid mesh)" : "");
    if (v & FEM_DEVERR_BADMESH)
        return fail(FEM_ERR_BADMESH, "a kernel met a vertex id outside [0, n_verts) or a cell with det J = 0 or "
                                     "a non-finite det J (fem_check_mesh counts them)");
    return FEM_OK;
}

extern "C" fem_status fem_selftest_wait(int64_t budget_ns, fem_stream stream) {
    if (budget_ns < 0 || budget_ns > int64_t(10) * 1000 * 1000 * 1000)
        return fail(FEM_ERR_ARG, "budget_ns must lie in [0, 10 s]");
    unsigned *w = device_error_word();
    if (!w) return fail(FEM_ERR_CUDA, "fem_selftest_wait: device error word unavailable");
    selftest_wait_kernel<<<1, 32, 0, stream>>>(static_cast<uint64_t>(budget_ns), w);
    return check_launch("fem_selftest_wait");
}

extern "C" fem_status fem_probe(int kind, int64_t n_threads, int iters, void *out, fem_stream stream) {
    if (kind < 0 || kind > 3) return fail(FEM_ERR_ARG, "probe kind %d", kind);
    if (n_threads <= 0 || n_threads % 256 != 0 || n_threads / 256 > 0x7fffffff)
        return fail(FEM_ERR_ARG, "n_threads must be a positive multiple of 256");
    if (iters < 0 || !out) return fail(FEM_ERR_ARG, "bad iters or NULL out");
    dim3 grid(static_cast<unsigned>(n_threads / 256));
    switch (kind) {
        case 0: probe_kernel<0><<<grid, 256, 0, stream>>>(iters, out); break;
        case 1: probe_kernel<1><<<grid, 256, 0, stream>>>(iters, out); break;
        case 2: probe_kernel<2><<<grid, 256, 0, stream>>>(iters, out); break;
        default: probe_kernel<3><<<grid, 256, 0, stream>>>(iters, out); break;
    }
    return check_launch("fem_probe");
}

extern "C" fem_status fem_set_mixed_threshold(double tau) {
    if (!(tau >= 0.0) || !std::isfinite(tau)) return fail(FEM_ERR_ARG, "tau must be finite and >= 0");
    g_mixed_tau.store(static_cast<float>(tau), std::memory_order_relaxed);
    return FEM_OK;
}

extern "C" double fem_get_mixed_threshold(void) { return static_cast<double>(mixed_tau()); }

extern "C" const char *fem_status_string(fem_status st) {
    switch (st) {
        case FEM_OK: return "FEM_OK";
        case FEM_ERR_ARG: return "FEM_ERR_ARG: bad argument";
        case FEM_ERR_SHAPE: return "FEM_ERR_SHAPE: unsupported size";
        case FEM_ERR_CUDA: return "FEM_ERR_CUDA: CUDA error";
        case FEM_ERR_OOM: return "FEM_ERR_OOM: buffer too small";
        case FEM_ERR_BADMESH: return "FEM_ERR_BADMESH: invalid mesh";
        case FEM_ERR_TIMEOUT: return "FEM_ERR_TIMEOUT: bounded wait expired";
        case FEM_ERR_UNSUPPORTED: return "FEM_ERR_UNSUPPORTED";
    }
    return "unknown fem_status";
}

extern "C" const char *fem_last_error(void) { return g_last_error; }

extern "C" const char *fem_version(void) { return "libfem 0.1 (sm_103a)"; }
