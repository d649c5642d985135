// fem_geometry.cu -- the paper's precomputed-geometry input layout (Sec. 3 and the
// Appendix: the integration kernel loads J^{-1} and det J per cell instead of computing
// them) as an alternate entry for the Laplacian residual.
//
//   fem_precompute_geometry       per cell: J^{-1} (row-major, d*d values) and det J,
//                                 computed once per mesh from the coordinates
//   fem_integrate_laplacian_geom  the Laplacian element residual from conn, u, K and the
//                                 precomputed geometry: no coordinate gathers, d*d + 1
//                                 more streamed values per cell
//
// With G_b = J^{-T} grad_ref phi_b (columns of J^{-T}: G_j = row j of J^{-1} for j >= 1,
// G_0 = -(G_1 + ... + G_d)) and g = sum_b u_b G_b:
//     r_b = (sum_q w_q K_q) |det J| G_b . g,  r_0 = -(r_1 + ... + r_d).
#include "fem_cell.cuh"

namespace fem {

struct GeomArgs {
    const double *X[3];
    const int32_t *conn;
    void *geom;  // [dim*dim + 1][C]: invJ rows then det J
    int64_t C;
    uint32_t V;
    unsigned *err;  // device error word (FEM_DEVERR_BADMESH)
};

// geometry of CPT consecutive cells per thread, computed in float64 and stored in the
// value type (float32 storage rounds each entry once)
template <int DIM, int P>
__global__ void __launch_bounds__(kBlock) geometry_kernel(const __grid_constant__ GeomArgs a) {
    pdl_wait();  // overlapped launch: the previous kernel's writes are visible from here
    pdl_trigger();
    constexpr int NB = DIM + 1;
    using T = val_t<P>;
    const int64_t C = a.C;
    T *geom = static_cast<T *>(a.geom);
    const double *X[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) X[k] = a.X[k];
    uint32_t vmax = 0;
    bool bad_det = false;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < C; c += stride) {
        uint32_t v[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) v[b] = clamp_vid(a.conn[b * C + c], a.V, vmax);
        double xs[NB][DIM], e[DIM][DIM], n[DIM][DIM];
        gather_coords<DIM>(X, v, xs);
        columns_f64<DIM>(xs, e);
        const double det = adjugate_rows<DIM>(e, n);
        bad_det |= det_bad(det) | ids_repeat<NB>(v);
        const double rdet = 1.0 / det;
        // (J^{-1})_{ji} = n_j[i] / det J  (row j of J^{-1} is n_j / det J)
#pragma unroll
        for (int j = 0; j < DIM; ++j)
#pragma unroll
            for (int i = 0; i < DIM; ++i) geom[(j * DIM + i) * C + c] = static_cast<T>(n[j][i] * rdet);
        geom[(DIM * DIM) * C + c] = static_cast<T>(det);
    }
    report_mesh(a.err, vmax, a.V, bad_det);
}

struct LapGeomArgs {
    const int32_t *conn;
    const void *u;
    const void *K;
    const void *geom;
    void *out;
    int64_t C;
    uint32_t V;
    unsigned *err;  // device error word (FEM_DEVERR_BADMESH)
    QuadW w;
};

template <int P>
__device__ __forceinline__ val_t<P> gweight(const QuadW &w, int q) {
    if constexpr (P == FEM_FP64) return w.wd[q];
    else return w.wf[q];
}

// One thread owns CPT consecutive cells (vector loads of every cell-indexed row). NQ > 0
// fixes the quadrature size at compile time.
template <int DIM, int P, int CPT, int NQ>
__global__ void __launch_bounds__(kBlock) lap_geom_kernel(const __grid_constant__ LapGeomArgs a) {
    pdl_wait();  // overlapped launch: the previous kernel's writes are visible from here
    pdl_trigger();
    constexpr int NB = DIM + 1;
    using T = val_t<P>;
    const int64_t C = a.C;
    const T *__restrict__ u = static_cast<const T *>(a.u);
    const T *__restrict__ K = static_cast<const T *>(a.K);
    const T *__restrict__ geom = static_cast<const T *>(a.geom);
    T *__restrict__ out = static_cast<T *>(a.out);
    const int nq = NQ > 0 ? NQ : a.w.nq;
    uint32_t vmax = 0;
    bool bad_det = false;
    const int64_t ngroups = (C + CPT - 1) / CPT;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < ngroups; g += stride) {
        const int64_t c0 = g * CPT;
        int32_t vid[NB][CPT];
#pragma unroll
        for (int b = 0; b < NB; ++b) load_row<CPT>(a.conn + b * C + c0, vid[b]);
        T gm[DIM * DIM + 1][CPT];
#pragma unroll
        for (int r = 0; r <= DIM * DIM; ++r) load_row<CPT>(geom + r * C + c0, gm[r]);
        qsum_t<P> ks[CPT];
#pragma unroll(NQ > 0 ? NQ : 1)
        for (int q = 0; q < nq; ++q) {
            T kq[CPT];
            load_row<CPT>(K + q * C + c0, kq);
#pragma unroll
            for (int i = 0; i < CPT; ++i) {
                if (q == 0) ks[i].first(gweight<P>(a.w, 0), kq[i]);
                else ks[i].add(gweight<P>(a.w, q), kq[i]);
            }
        }
        T r[NB][CPT];
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            T uu[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) uu[b] = ld_gather(u + clamp_vid(vid[b][i], a.V, vmax));
            // g = sum_{j>=1} (u_j - u_0) G_j, G_j = row j of J^{-1}
            T gv[DIM];
#pragma unroll
            for (int k = 0; k < DIM; ++k) gv[k] = zero<T>();
#pragma unroll
            for (int j = 0; j < DIM; ++j) {
                const T du = uu[j + 1] - uu[0];
#pragma unroll
                for (int k = 0; k < DIM; ++k) gv[k] = fma(du, gm[j * DIM + k][i], gv[k]);
            }
            T det = gm[DIM * DIM][i];
            bad_det |= det_bad(det);
            det = det < T(0) ? -det : det;
            const T s = ks[i].value() * det;
            T sum = zero<T>();
#pragma unroll
            for (int j = 0; j < DIM; ++j) {
                T d = gm[j * DIM][i] * gv[0];
#pragma unroll
                for (int k = 1; k < DIM; ++k) d = fma(gm[j * DIM + k][i], gv[k], d);
                r[j + 1][i] = s * d;
                sum = sum + r[j + 1][i];
            }
            r[0][i] = -sum;
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) store_row<CPT>(out + b * C + c0, r[b]);
    }
    report_mesh(a.err, vmax, a.V, bad_det);
}

template <int DIM, int P>
static fem_status launch_geom_lap(const LapGeomArgs &a, bool vec, cudaStream_t s) {
    if (vec && a.w.nq == DIM + 1) {
        // one wave of resident CTAs (24.5 against 24.7 us per step with up to 8 waves)
        auto k = lap_geom_kernel<DIM, P, 4, DIM + 1>;
        launch_overlapped(k, resident_grid(reinterpret_cast<const void *>(k), kBlock, (a.C + 3) / 4), kBlock, 0, s, a);
    } else if (vec) {
        auto k = lap_geom_kernel<DIM, P, 4, 0>;
        launch_overlapped(k, grid_for((a.C + 3) / 4, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, s, a);
    } else {
        auto k = lap_geom_kernel<DIM, P, 1, 0>;
        launch_overlapped(k, grid_for(a.C, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, s, a);
    }
    return check_launch("fem_integrate_laplacian_geom");
}

}  // namespace fem

using namespace fem;

extern "C" fem_status fem_precompute_geometry(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                              const int32_t *conn, void *geom, fem_precision prec,
                                              fem_stream stream) {
    fem_status st = check_common(dim, n_cells, n_verts, coords, conn);
    if (st != FEM_OK) return st;
    if (prec != FEM_FP64 && prec != FEM_FP32_MIXED && prec != FEM_FP32)
        return fail(FEM_ERR_ARG, "unknown precision %d", static_cast<int>(prec));
    if (n_cells == 0) return FEM_OK;
    if (!geom) return fail(FEM_ERR_ARG, "geom is NULL");
    GeomArgs a;
    for (int k = 0; k < 3; ++k) a.X[k] = coords + (k < dim ? k : 0) * n_verts;
    a.conn = conn;
    a.geom = geom;
    a.C = n_cells;
    a.V = static_cast<uint32_t>(n_verts);
    if (!(a.err = device_error_word())) return fail(FEM_ERR_CUDA, "device error word unavailable");
    const bool f64 = prec == FEM_FP64;
    if (dim == 2) {
        auto k = f64 ? geometry_kernel<2, FEM_FP64> : geometry_kernel<2, FEM_FP32>;
        launch_overlapped(k, grid_for(n_cells, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, stream, a);
    } else {
        auto k = f64 ? geometry_kernel<3, FEM_FP64> : geometry_kernel<3, FEM_FP32>;
        launch_overlapped(k, grid_for(n_cells, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, stream, a);
    }
    return check_launch("fem_precompute_geometry");
}

extern "C" fem_status fem_integrate_laplacian_geom(int dim, int64_t n_cells, int64_t n_verts, const int32_t *conn,
                                                   const void *u, const void *K, int n_q, const double *qpts,
                                                   const double *qw, const void *geom, void *elem_out,
                                                   fem_precision prec, fem_stream stream) {
    if (dim != 2 && dim != 3) return fail(FEM_ERR_ARG, "dim = %d, must be 2 or 3", dim);
    if (n_cells < 0 || n_verts < 0) return fail(FEM_ERR_ARG, "negative size");
    if (n_cells > 0 && n_verts < 1) return fail(FEM_ERR_SHAPE, "cells without vertices");
    if ((dim * dim + 1) * n_cells >= (int64_t(1) << 31) || n_verts >= (int64_t(1) << 31))
        return fail(FEM_ERR_SHAPE, "mesh too large for int32 indexing");
    if (prec != FEM_FP64 && prec != FEM_FP32_MIXED && prec != FEM_FP32)
        return fail(FEM_ERR_ARG, "unknown precision %d", static_cast<int>(prec));
    LapGeomArgs a;
    fem_status st = load_quadrature(dim, n_q, qpts, qw, a.w);
    if (st != FEM_OK) return st;
    if (n_cells == 0) return FEM_OK;
    if (!conn || !u || !K || !geom || !elem_out) return fail(FEM_ERR_ARG, "a NULL array argument");
    a.conn = conn;
    a.u = u;
    a.K = K;
    a.geom = geom;
    a.out = elem_out;
    a.C = n_cells;
    a.V = static_cast<uint32_t>(n_verts);
    if (!(a.err = device_error_word())) return fail(FEM_ERR_CUDA, "device error word unavailable");
    const bool vec = n_cells % 4 == 0 && aligned16(conn) && aligned16(K) && aligned16(geom) && aligned16(elem_out);
    // the float32 forms both integrate from float32 geometry (there are no coordinates
    // to fall back on): FEM_FP32_MIXED differs from FEM_FP32 only in its compensated sum
    switch (dim * 10 + static_cast<int>(prec)) {
        case 20: return launch_geom_lap<2, FEM_FP64>(a, vec, stream);
        case 21: return launch_geom_lap<2, FEM_FP32_MIXED>(a, vec, stream);
        case 22: return launch_geom_lap<2, FEM_FP32>(a, vec, stream);
        case 30: return launch_geom_lap<3, FEM_FP64>(a, vec, stream);
        case 31: return launch_geom_lap<3, FEM_FP32_MIXED>(a, vec, stream);
        case 32: return launch_geom_lap<3, FEM_FP32>(a, vec, stream);
    }
    return fail(FEM_ERR_ARG, "unsupported dim/precision");
}
