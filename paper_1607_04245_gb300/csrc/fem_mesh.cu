// fem_mesh.cu -- vertex-to-cell lists (the transpose of the connectivity, i.e. the
// assembly operator E of Eq. 2 as lists), the deterministic nodal gather E^T applied
// to element vectors, and the mesh validation pass.
#include "fem_cell.cuh"

namespace fem {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

static int64_t scan_tiles_for(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

// ------------------------------------------------------------------ scan (three passes)

// Exclusive prefix sum of x over the CTA (kScanThreads threads); the CTA total is
// stored to *total (shared memory) and is visible to every thread on return.
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t x, int32_t *total) {
    constexpr int kWarps = kScanThreads / 32;
    __shared__ int32_t warp_off[kWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_off[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int32_t t = lane < kWarps ? warp_off[lane] : 0;
        int32_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < kWarps) warp_off[lane] = ti - t;
        if (lane == 31) *total = ti;
    }
    __syncthreads();
    const int32_t off = warp_off[wid];
    __syncthreads();  // warp_off may be reused by the next call
    return off + incl - x;
}

// in-place inclusive scan of one tile; the tile's total goes to tile_sums[tile]
__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(int32_t *data, int64_t n, int32_t *tile_sums) {
    __shared__ int32_t s_total;
    const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanItems;
    int32_t v[kScanItems];
    int32_t run = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        run += (base + i < n) ? data[base + i] : 0;
        v[i] = run;  // inclusive within the thread
    }
    const int32_t off = block_exclusive_scan(run, &s_total);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) data[base + i] = v[i] + off;
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = s_total;
}

// exclusive scan of the tile sums in place (one CTA, chunks of a tile with a carry)
__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(int32_t *sums, int64_t n) {
    __shared__ int32_t s_total;
    int32_t carry = 0;
    for (int64_t c = 0; c < n; c += kScanTile) {
        const int64_t base = c + int64_t(threadIdx.x) * kScanItems;
        int32_t v[kScanItems], run = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            v[i] = run;  // exclusive within the thread
            run += (base + i < n) ? sums[base + i] : 0;
        }
        const int32_t off = block_exclusive_scan(run, &s_total);
#pragma unroll
        for (int i = 0; i < kScanItems; ++i)
            if (base + i < n) sums[base + i] = carry + off + v[i];
        carry += s_total;
        __syncthreads();
    }
}

__global__ void add_offsets_kernel(int32_t *data, int64_t n, const int32_t *tile_sums) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) data[i] += tile_sums[i / kScanTile];
}

// inclusive scan of data[0..n) with workspace tile_sums[scan_tiles_for(n)]
static fem_status inclusive_scan(int32_t *data, int64_t n, int32_t *tile_sums, cudaStream_t s) {
    if (n == 0) return FEM_OK;
    const int64_t tiles = scan_tiles_for(n);
    scan_tiles_kernel<<<static_cast<unsigned>(tiles), kScanThreads, 0, s>>>(data, n, tile_sums);
    scan_sums_kernel<<<1, kScanThreads, 0, s>>>(tile_sums, tiles);
    add_offsets_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(data, n, tile_sums);
    return check_launch("scan");
}

// ------------------------------------------------------------------ vertex-to-cell lists

__global__ void count_kernel(const int32_t *conn, int64_t total, uint32_t V, int32_t *ptr1, unsigned *err) {
    uint32_t vmax = 0;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < total; j += stride)
        atomicAdd(ptr1 + clamp_vid(conn[j], V, vmax), 1);
    report_mesh(err, vmax, V, false);
}

__global__ void copy_kernel(const int32_t *src, int32_t *dst, int64_t n) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

template <int NB>
__global__ void fill_kernel(const int32_t *conn, int64_t C, uint32_t V, int32_t *cursor, int32_t *idx) {
    const int a = blockIdx.y;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < C; e += stride) {
        const uint32_t v = clamp_vid(conn[a * C + e], V);
        const int32_t pos = atomicAdd(cursor + v, 1);
        idx[pos] = static_cast<int32_t>(e * NB + a);
    }
}

// per-vertex insertion sort: the list order becomes cell order, independent of the
// order in which the atomics above landed. Lists of up to kSortLocal entries (every
// vertex of the workloads' meshes: 6 in 2D, up to 24 in 3D) are sorted in a per-thread
// array and written back once; longer ones in place.
constexpr int kSortLocal = 32;

__global__ void sort_segments_kernel(const int32_t *ptr, int32_t *idx, int64_t V) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; n < V; n += stride) {
        const int32_t b = ptr[n], e = ptr[n + 1];
        if (e - b <= kSortLocal) {
            int32_t t[kSortLocal];
            const int m = e - b;
            for (int i = 0; i < m; ++i) t[i] = idx[b + i];
            for (int i = 1; i < m; ++i) {
                const int32_t x = t[i];
                int j = i - 1;
                while (j >= 0 && t[j] > x) {
                    t[j + 1] = t[j];
                    --j;
                }
                t[j + 1] = x;
            }
            for (int i = 0; i < m; ++i) idx[b + i] = t[i];
            continue;
        }
        for (int32_t i = b + 1; i < e; ++i) {
            int32_t x = idx[i], j = i - 1;
            while (j >= b && idx[j] > x) {
                idx[j + 1] = idx[j];
                --j;
            }
            idx[j + 1] = x;
        }
    }
}

// ------------------------------------------------------------------ nodal gather


template <int NB, int NCOMP, class T>
__global__ void gather_kernel(int64_t C, int64_t V, const T *__restrict__ elem, const int32_t *__restrict__ ptr,
                              const int32_t *__restrict__ idx, T *__restrict__ out) {
    pdl_wait();  // overlapped launch: the previous kernel's writes are visible from here
    pdl_trigger();
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    auto entry = [&](int32_t t, int k) {
        const int32_t cell = t / NB, a = t - cell * NB;
        return __ldg(elem + int64_t(a * NCOMP + k) * C + cell);
    };
    for (int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; n < V; n += stride) {
        const int32_t b = ptr[n], e = ptr[n + 1];
        NodeSum<T> acc[NCOMP];
        // kGatherBatch list entries at a time: their loads are independent and in flight
        // together; the sums still take the entries one by one in list order. (A warp
        // reading 32 vertices' lists together with coalesced loads and summing from shared
        // memory was slower: 60.4 against 48.8 us for the adjoint on 1,572,864 tets.)
        int32_t j = b;
        for (; j + kGatherBatch <= e; j += kGatherBatch) {
            int32_t t[kGatherBatch];
            T val[kGatherBatch][NCOMP];
#pragma unroll
            for (int i = 0; i < kGatherBatch; ++i) t[i] = __ldg(idx + j + i);
#pragma unroll
            for (int i = 0; i < kGatherBatch; ++i)
#pragma unroll
                for (int k = 0; k < NCOMP; ++k) val[i][k] = entry(t[i], k);
#pragma unroll
            for (int i = 0; i < kGatherBatch; ++i)
#pragma unroll
                for (int k = 0; k < NCOMP; ++k) acc[k].add(val[i][k]);
        }
        for (; j < e; ++j) {
            const int32_t t = __ldg(idx + j);
#pragma unroll
            for (int k = 0; k < NCOMP; ++k) acc[k].add(entry(t, k));
        }
#pragma unroll
        for (int k = 0; k < NCOMP; ++k) out[k * V + n] = acc[k].value();
    }
}

template <int NB, class T>
static void launch_gather_t(int n_comp, int64_t C, int64_t V, const void *elem, const int32_t *ptr,
                            const int32_t *idx, void *out, cudaStream_t s) {
    const T *el = static_cast<const T *>(elem);
    T *o = static_cast<T *>(out);
    switch (n_comp) {
        case 1: {
            auto k = gather_kernel<NB, 1, T>;
            launch_overlapped(k, grid_for(V, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, s, C, V, el, ptr, idx, o);
        } break;
        case 2: {
            auto k = gather_kernel<NB, 2, T>;
            launch_overlapped(k, grid_for(V, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, s, C, V, el, ptr, idx, o);
        } break;
        default: {
            auto k = gather_kernel<NB, 3, T>;
            launch_overlapped(k, grid_for(V, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, s, C, V, el, ptr, idx, o);
        } break;
    }
}

fem_status launch_gather(int dim, int n_comp, int64_t C, int64_t V, const void *elem, const int32_t *node_ptr,
                         const int32_t *node_idx, void *out, fem_precision prec, cudaStream_t s) {
    if (V == 0) return FEM_OK;
    const bool f64 = prec == FEM_FP64 || prec == FEM_FP64_DF;  // float64 values either way
    if (dim == 2) {
        if (f64) launch_gather_t<3, double>(n_comp, C, V, elem, node_ptr, node_idx, out, s);
        else launch_gather_t<3, float>(n_comp, C, V, elem, node_ptr, node_idx, out, s);
    } else {
        if (f64) launch_gather_t<4, double>(n_comp, C, V, elem, node_ptr, node_idx, out, s);
        else launch_gather_t<4, float>(n_comp, C, V, elem, node_ptr, node_idx, out, s);
    }
    return check_launch("nodal gather");
}

// ------------------------------------------------------------------ mesh validation

template <int DIM>
__global__ void check_mesh_kernel(const double *X0, int64_t C, uint32_t V, const int32_t *conn, float tau2,
                                  unsigned long long *counts) {
    constexpr int NB = DIM + 1;
    __shared__ unsigned long long s_cnt[4];
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long c_bad = 0, c_degen = 0, c_fallback = 0, c_neg = 0;
    const double *X[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) X[k] = X0 + int64_t(k) * V;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < C; c += stride) {
        uint32_t v[NB];
        bool ids_ok = true;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            int32_t id = conn[b * C + c];
            if (id < 0 || static_cast<uint32_t>(id) >= V) ++c_bad, ids_ok = false;
            v[b] = clamp_vid(id, V);
        }
        if (!ids_ok) continue;
        double xs[NB][DIM], e[DIM][DIM], n[DIM][DIM];
        gather_coords<DIM>(X, v, xs);
        columns_f64<DIM>(xs, e);
        double det = adjugate_rows<DIM>(e, n);
        // degenerate to rounding: |det J| <= 16 eps_64 prod_j |e_j| (FMA contraction can
        // leave a rounding residue instead of an exact zero for repeated vertices)
        double pn = 1.0;
#pragma unroll
        for (int j = 0; j < DIM; ++j) pn *= sqrt(dotv<DIM>(e[j], e[j]));
        const bool degenerate = !(fabs(det) > 16.0 * DBL_EPSILON * pn) || !isfinite(det);
        if (degenerate) ++c_degen;
        else if (det < 0.0) ++c_neg;
        float ef[DIM][DIM], nf[DIM][DIM];
        columns_mixed<DIM>(xs, ef);
        float detf = adjugate_rows<DIM>(ef, nf);
        if (!shape_ok<DIM>(ef, detf, tau2)) ++c_fallback;
    }
    atomicAdd(&s_cnt[0], c_bad);
    atomicAdd(&s_cnt[1], c_degen);
    atomicAdd(&s_cnt[2], c_fallback);
    atomicAdd(&s_cnt[3], c_neg);
    __syncthreads();
    if (threadIdx.x < 4 && s_cnt[threadIdx.x]) atomicAdd(counts + threadIdx.x, s_cnt[threadIdx.x]);
}

}  // namespace fem

using namespace fem;

extern "C" int64_t fem_node2cell_work_size(int64_t n_verts) {
    if (n_verts < 0) return 0;
    return n_verts + scan_tiles_for(n_verts) + 1;
}

extern "C" fem_status fem_build_node2cell(int dim, int64_t n_cells, int64_t n_verts, const int32_t *conn,
                                          int32_t *node_ptr, int32_t *node_idx, int32_t *work, fem_stream stream) {
    if (dim != 2 && dim != 3) return fail(FEM_ERR_ARG, "dim = %d, must be 2 or 3", dim);
    if (n_cells < 0 || n_verts < 0) return fail(FEM_ERR_ARG, "negative size");
    if ((dim + 1) * n_cells >= (int64_t(1) << 31) || n_verts >= (int64_t(1) << 31))
        return fail(FEM_ERR_SHAPE, "mesh too large for int32 indexing");
    if (n_cells > 0 && (n_verts < 1 || !conn)) return fail(FEM_ERR_ARG, "cells without vertices or NULL conn");
    fem_status st;
    if (!node_ptr || (n_verts > 0 && !work) || (n_cells > 0 && !node_idx))
        return fail(FEM_ERR_ARG, "node_ptr, node_idx or work is NULL");
    const int NB = dim + 1;
    cudaStream_t s = stream;
    if (cudaMemsetAsync(node_ptr, 0, sizeof(int32_t) * (n_verts + 1), s) != cudaSuccess)
        return check_launch("node2cell memset");
    if (n_cells == 0 || n_verts == 0) return check_launch("node2cell");
    const uint32_t V = static_cast<uint32_t>(n_verts);
    unsigned *err = device_error_word();
    if (!err) return fail(FEM_ERR_CUDA, "device error word unavailable");
    count_kernel<<<grid_for(NB * n_cells, kBlock, reinterpret_cast<const void *>(count_kernel)), kBlock, 0, s>>>(
        conn, NB * n_cells, V, node_ptr + 1, err);
    if ((st = inclusive_scan(node_ptr + 1, n_verts, work + n_verts, s)) != FEM_OK) return st;
    copy_kernel<<<grid_for(n_verts, kBlock, reinterpret_cast<const void *>(copy_kernel)), kBlock, 0, s>>>(
        node_ptr, work, n_verts);
    dim3 fgrid(grid_for(n_cells, kBlock, reinterpret_cast<const void *>(fill_kernel<4>)), NB);
    if (dim == 2) fill_kernel<3><<<fgrid, kBlock, 0, s>>>(conn, n_cells, V, work, node_idx);
    else fill_kernel<4><<<fgrid, kBlock, 0, s>>>(conn, n_cells, V, work, node_idx);
    sort_segments_kernel<<<grid_for(n_verts, kBlock, reinterpret_cast<const void *>(sort_segments_kernel)), kBlock,
                           0, s>>>(node_ptr, node_idx, n_verts);
    return check_launch("fem_build_node2cell");
}

extern "C" fem_status fem_gather_nodes(int dim, int n_comp, int64_t n_cells, int64_t n_verts, const void *elem,
                                       const int32_t *node_ptr, const int32_t *node_idx, void *out,
                                       fem_precision prec, fem_stream stream) {
    if (dim != 2 && dim != 3) return fail(FEM_ERR_ARG, "dim = %d", dim);
    if (n_comp < 1 || n_comp > 3) return fail(FEM_ERR_ARG, "n_comp = %d", n_comp);
    if (n_cells < 0 || n_verts < 0) return fail(FEM_ERR_ARG, "negative size");
    if (prec != FEM_FP64 && prec != FEM_FP32_MIXED && prec != FEM_FP32 && prec != FEM_FP64_DF)
        return fail(FEM_ERR_ARG, "unknown precision %d", static_cast<int>(prec));
    if (n_verts > 0 && (!node_ptr || !out)) return fail(FEM_ERR_ARG, "NULL argument");
    if (n_cells > 0 && (!elem || !node_idx)) return fail(FEM_ERR_ARG, "NULL argument");
    return launch_gather(dim, n_comp, n_cells, n_verts, elem, node_ptr, node_idx, out, prec, stream);
}

extern "C" fem_status fem_check_mesh(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                     const int32_t *conn, int64_t *counts, fem_stream stream) {
    fem_status st = check_common(dim, n_cells, n_verts, coords, conn);
    if (st != FEM_OK) return st;
    if (!counts) return fail(FEM_ERR_ARG, "counts is NULL");
    if (cudaMemsetAsync(counts, 0, 4 * sizeof(int64_t), stream) != cudaSuccess) return check_launch("check memset");
    if (n_cells == 0) return check_launch("fem_check_mesh");
    float tau = mixed_tau();
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(counts);
    const uint32_t V = static_cast<uint32_t>(n_verts);
    if (dim == 2) {
        auto k = check_mesh_kernel<2>;
        k<<<grid_for(n_cells, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, stream>>>(coords, n_cells, V,
                                                                                              conn, tau * tau, cnt);
    } else {
        auto k = check_mesh_kernel<3>;
        k<<<grid_for(n_cells, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, stream>>>(coords, n_cells, V,
                                                                                              conn, tau * tau, cnt);
    }
    return check_launch("fem_check_mesh");
}
