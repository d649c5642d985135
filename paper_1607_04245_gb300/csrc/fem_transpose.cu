// fem_transpose.cu -- the paper's thread-transposition kernel (Sec. 3, Figs. 1-3) rebuilt
// for GB300 as an ablation beside the per-cell kernels of fem_laplacian.cu.
//
// The paper's scheme: a thread block integrates batches of cells. Inputs are the paper's
// precomputed, element-local data: J^{-1} and det J per cell (fem_precompute_geometry)
// and the element basis coefficients u_e (fem_element_values, the closure of u). Per batch
// of B cells:
//   1. the batch's geometry, coefficients and K_q are loaded into shared memory;
//   2. quadrature phase (Sec. 3.1): one thread per (cell, q) evaluates grad u at xi_q from
//      the tabulated reference derivatives, applies f1 = K_q grad u, scales by w_q |det J|
//      and stores f1 in shared memory;
//   3. one barrier; basis phase (Sec. 3.2): one thread per (cell, b) contracts
//      G_b(q) . f1(q) over q and writes the element vector entry.
// A CTA runs `batches` batches one after the other (the paper's N_cb); B cells per batch
// corresponds to the paper's N_bl blocks of N_bs = LCM(N_b, N_q) cells. With the rules
// used here N_q = N_b, so both phases keep B * N_b threads busy.
//
// Differences from the paper's listing: value arrays are structure-of-arrays with the
// cell index fastest (every phase's loads and stores are coalesced with the thread ->
// (q or b, cell) mapping below) instead of per-cell arrays, and the reference gradients
// are passed in the launch parameters.
#include "fem_cell.cuh"

namespace fem {

struct TrArgs {
    const void *ue;    // [NB][C] element basis coefficients
    const void *K;     // [NQ][C]
    const void *geom;  // [d*d + 1][C]: J^{-1} rows, det J
    void *out;         // [NB][C]
    int64_t C;
    double wd[4];
    float wf[4];
    double dphid[4][4][3];  // reference gradients at each quadrature point
    float dphif[4][4][3];
};

template <int DIM, class T, int B>
__global__ void __launch_bounds__(B *(DIM + 1)) transpose_kernel(const __grid_constant__ TrArgs a, int batches) {
    constexpr int NB = DIM + 1, NQ = DIM + 1, NG = DIM * DIM + 1;
    __shared__ T s_geom[NG][B];
    __shared__ T s_ue[NB][B];
    __shared__ T s_K[NQ][B];
    __shared__ T s_f1[NQ][DIM][B];
    const T *ue = static_cast<const T *>(a.ue);
    const T *K = static_cast<const T *>(a.K);
    const T *geom = static_cast<const T *>(a.geom);
    T *out = static_cast<T *>(a.out);
    const int64_t C = a.C;
    const int t = threadIdx.x;
    const int slot = t / B, c = t % B;  // (q or b, cell within the batch)
    for (int batch = 0; batch < batches; ++batch) {
        const int64_t c0 = (int64_t(blockIdx.x) * batches + batch) * B;
        if (c0 >= C) break;
        const int n = static_cast<int>(C - c0 < B ? C - c0 : B);
        // 1. coalesced loads of the batch into shared memory
        for (int i = t; i < NG * B; i += B * NB) {
            const int r = i / B, j = i % B;
            s_geom[r][j] = j < n ? geom[r * C + c0 + j] : T(0);
        }
        for (int i = t; i < NB * B; i += B * NB) {
            const int r = i / B, j = i % B;
            s_ue[r][j] = j < n ? ue[r * C + c0 + j] : T(0);
            s_K[r][j] = j < n ? K[r * C + c0 + j] : T(0);
        }
        __syncthreads();
        // 2. quadrature phase: thread (q = slot, cell c)
        {
            const int q = slot;
            T g[DIM];
#pragma unroll
            for (int i = 0; i < DIM; ++i) g[i] = T(0);
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                // G_b(q) = J^{-T} grad_ref phi_b(xi_q):  G_i = sum_k invJ[k][i] dphi[k]
#pragma unroll
                for (int i = 0; i < DIM; ++i) {
                    T Gi = T(0);
#pragma unroll
                    for (int k = 0; k < DIM; ++k) {
                        const T dp = std::is_same<T, double>::value ? T(a.dphid[q][b][k]) : T(a.dphif[q][b][k]);
                        Gi = fma(s_geom[k * DIM + i][c], dp, Gi);
                    }
                    g[i] = fma(s_ue[b][c], Gi, g[i]);
                }
            }
            T det = s_geom[DIM * DIM][c];
            det = det < T(0) ? -det : det;
            const T wq = std::is_same<T, double>::value ? T(a.wd[q]) : T(a.wf[q]);
            const T s = s_K[q][c] * wq * det;
#pragma unroll
            for (int i = 0; i < DIM; ++i) s_f1[q][i][c] = s * g[i];
        }
        __syncthreads();
        // 3. basis phase: thread (b = slot, cell c)
        {
            const int b = slot;
            T r = T(0);
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
#pragma unroll
                for (int i = 0; i < DIM; ++i) {
                    T Gi = T(0);
#pragma unroll
                    for (int k = 0; k < DIM; ++k) {
                        const T dp = std::is_same<T, double>::value ? T(a.dphid[q][b][k]) : T(a.dphif[q][b][k]);
                        Gi = fma(s_geom[k * DIM + i][c], dp, Gi);
                    }
                    r = fma(Gi, s_f1[q][i][c], r);
                }
            }
            if (c < n) __stcs(out + b * C + c0 + c, r);
        }
        __syncthreads();  // shared memory is reused by the next batch
    }
}

// element basis coefficients: ue[b][e] = u[conn[b][e]] (the closure of u)
template <class T>
__global__ void element_values_kernel(int64_t total, int64_t C, uint32_t V, const int32_t *conn, const T *u, T *ue,
                                      unsigned *err) {
    uint32_t vmax = 0;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += stride)
        ue[i] = ld_gather(u + clamp_vid(conn[i], V, vmax));
    report_mesh(err, vmax, V, false);
}

template <int DIM, class T, int B>
static fem_status launch_tr(const TrArgs &a, int batches, cudaStream_t s) {
    const int64_t per = int64_t(B) * batches;
    const int64_t grid = (a.C + per - 1) / per;
    if (grid > 0x7fffffff) return fail(FEM_ERR_SHAPE, "too many thread blocks");
    transpose_kernel<DIM, T, B><<<static_cast<unsigned>(grid), B * (DIM + 1), 0, s>>>(a, batches);
    return check_launch("fem_integrate_laplacian_transposed");
}

template <int DIM, class T>
static fem_status dispatch_tr(const TrArgs &a, int cells_per_batch, int batches, cudaStream_t s) {
    switch (cells_per_batch) {
        case 32: return launch_tr<DIM, T, 32>(a, batches, s);
        case 64: return launch_tr<DIM, T, 64>(a, batches, s);
        case 128: return launch_tr<DIM, T, 128>(a, batches, s);
        case 256:
            // float64 batches of 256 cells would exceed 48 KB of static shared memory
            if constexpr (sizeof(T) == 4) return launch_tr<DIM, T, 256>(a, batches, s);
            break;
    }
    return fail(FEM_ERR_ARG, "cells_per_batch = %d, must be 32, 64, 128 or (float32 forms) 256", cells_per_batch);
}

}  // namespace fem

using namespace fem;

extern "C" fem_status fem_element_values(int dim, int64_t n_cells, int64_t n_verts, const int32_t *conn, const void *u,
                                         void *ue, fem_precision prec, fem_stream stream) {
    if (dim != 2 && dim != 3) return fail(FEM_ERR_ARG, "dim = %d, must be 2 or 3", dim);
    if (n_cells < 0 || n_verts < 0) return fail(FEM_ERR_ARG, "negative size");
    if ((dim + 1) * n_cells >= (int64_t(1) << 31) || n_verts >= (int64_t(1) << 31))
        return fail(FEM_ERR_SHAPE, "mesh too large for int32 indexing");
    if (prec != FEM_FP64 && prec != FEM_FP32_MIXED && prec != FEM_FP32)
        return fail(FEM_ERR_ARG, "unknown precision %d", static_cast<int>(prec));
    if (n_cells == 0) return FEM_OK;
    if (n_verts < 1 || !conn || !u || !ue) return fail(FEM_ERR_ARG, "a NULL array argument or no vertices");
    const int64_t total = int64_t(dim + 1) * n_cells;
    unsigned *err = device_error_word();
    if (!err) return fail(FEM_ERR_CUDA, "device error word unavailable");
    if (prec == FEM_FP64) {
        auto k = element_values_kernel<double>;
        k<<<grid_for(total, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, stream>>>(
            total, n_cells, static_cast<uint32_t>(n_verts), conn, static_cast<const double *>(u),
            static_cast<double *>(ue), err);
    } else {
        auto k = element_values_kernel<float>;
        k<<<grid_for(total, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, stream>>>(
            total, n_cells, static_cast<uint32_t>(n_verts), conn, static_cast<const float *>(u),
            static_cast<float *>(ue), err);
    }
    return check_launch("fem_element_values");
}

extern "C" fem_status fem_integrate_laplacian_transposed(int dim, int64_t n_cells, const void *ue, const void *K,
                                                         int n_q, const double *qpts, const double *qw,
                                                         const void *geom, void *elem_out, int cells_per_batch,
                                                         int batches_per_block, fem_precision prec,
                                                         fem_stream stream) {
    if (dim != 2 && dim != 3) return fail(FEM_ERR_ARG, "dim = %d, must be 2 or 3", dim);
    if (n_cells < 0) return fail(FEM_ERR_ARG, "negative size");
    if ((dim * dim + 1) * n_cells >= (int64_t(1) << 31)) return fail(FEM_ERR_SHAPE, "mesh too large");
    if (prec != FEM_FP64 && prec != FEM_FP32_MIXED && prec != FEM_FP32)
        return fail(FEM_ERR_ARG, "unknown precision %d", static_cast<int>(prec));
    if (n_q != dim + 1)
        return fail(FEM_ERR_UNSUPPORTED, "the transposed kernel is built for n_q = dim + 1 = N_b (got %d)", n_q);
    if (!qpts || !qw) return fail(FEM_ERR_ARG, "qpts and qw are required");
    if (batches_per_block < 1) return fail(FEM_ERR_ARG, "batches_per_block must be >= 1");
    if (n_cells == 0) return FEM_OK;
    if (!ue || !K || !geom || !elem_out) return fail(FEM_ERR_ARG, "a NULL array argument");
    TrArgs a;
    a.ue = ue;
    a.K = K;
    a.geom = geom;
    a.out = elem_out;
    a.C = n_cells;
    for (int q = 0; q < 4; ++q) {
        a.wd[q] = q < n_q ? qw[q] : 0.0;
        a.wf[q] = static_cast<float>(a.wd[q]);
        for (int b = 0; b < 4; ++b)
            for (int k = 0; k < 3; ++k) {
                // P1 reference gradients (the same at every point): phi_0 = 1 - sum xi, phi_b = xi_{b-1}
                double v = 0.0;
                if (k < dim && b <= dim) v = b == 0 ? -1.0 : (k == b - 1 ? 1.0 : 0.0);
                a.dphid[q][b][k] = v;
                a.dphif[q][b][k] = static_cast<float>(v);
            }
    }
    if (dim == 2) return prec == FEM_FP64 ? dispatch_tr<2, double>(a, cells_per_batch, batches_per_block, stream)
                                          : dispatch_tr<2, float>(a, cells_per_batch, batches_per_block, stream);
    return prec == FEM_FP64 ? dispatch_tr<3, double>(a, cells_per_batch, batches_per_block, stream)
                            : dispatch_tr<3, float>(a, cells_per_batch, batches_per_block, stream);
}
