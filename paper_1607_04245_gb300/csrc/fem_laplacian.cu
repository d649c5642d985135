// fem_laplacian.cu -- element residual of the variable-coefficient Laplacian and the
// element part of its adjoint.
//
// Residual (Eq. 2, f0 = 0, f1 = K grad u). For P1 the gradient g = grad u is constant
// on a cell, so the quadrature phase (Sec. 3.1) and the basis phase (Sec. 3.2) reduce to
//     r_b = sum_q w_q |det J| K_q G_b . g = (Kbar / |det J|) n_b . h,
//     Kbar = sum_q w_q K_q,   h = sum_{j>=1} (u_j - u_0) n_j  (= det J * g),
// with n_b the adjugate rows (fem_cell.cuh) and n_0 = -(n_1 + ... + n_d); the code
// writes r_0 = -(r_1 + ... + r_d), which keeps every element sum at zero.
//
// Adjoint of J = sum_e lambda_e . r_e (not in the paper):
//     dJ/dK_{e,q}  = w_q |det J| (sum_b lambda_b G_b) . g = w_q (h_lambda . h_u) / |det J|
//     dJ/du_{e,a}  = (Kbar / |det J|) n_a . h_lambda   (the residual of the field lambda_e)
// The second is written per element to scratch and summed per vertex afterwards.
#include "fem_cell.cuh"

namespace fem {

struct LapArgs {
    const double *X[3];  // coordinate rows: X[k] = coords + k * V
    const int32_t *conn;
    const void *u;
    const void *K;
    const void *lam;  // adjoint weights [dim+1][C] (adjoint kernel only)
    void *out;        // residual [dim+1][C] or per-element dJ/du [dim+1][C]
    void *dK;         // [n_q][C] (adjoint kernel only)
    int64_t C;
    uint32_t V;
    float tau2;
    QuadW w;
};

// r_b from the adjugate rows, the determinant, the nodal values and Kbar.
template <int DIM, class T>
__device__ __forceinline__ void lap_element(const T (&n)[DIM][DIM], T det, const T (&uu)[DIM + 1], T kbar,
                                            T (&r)[DIM + 1]) {
    T h[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) h[i] = T(0);
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        T du = uu[j + 1] - uu[0];
#pragma unroll
        for (int i = 0; i < DIM; ++i) h[i] = fma(du, n[j][i], h[i]);
    }
    T s;
    if constexpr (std::is_same<T, double>::value) s = kbar / fabs(det);
    else s = __fdividef(kbar, fabsf(det));
    T sum = T(0);
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        r[j + 1] = s * dotv<DIM>(n[j], h);
        sum += r[j + 1];
    }
    r[0] = -sum;
}

// h_lambda . h_u / |det J|
template <int DIM, class T>
__device__ __forceinline__ T lap_dk_factor(const T (&n)[DIM][DIM], T det, const T (&uu)[DIM + 1],
                                           const T (&ll)[DIM + 1]) {
    T hu[DIM], hl[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) hu[i] = T(0), hl[i] = T(0);
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        T du = uu[j + 1] - uu[0], dl = ll[j + 1] - ll[0];
#pragma unroll
        for (int i = 0; i < DIM; ++i) hu[i] = fma(du, n[j][i], hu[i]), hl[i] = fma(dl, n[j][i], hl[i]);
    }
    T t = dotv<DIM>(hl, hu);
    if constexpr (std::is_same<T, double>::value) return t / fabs(det);
    else return __fdividef(t, fabsf(det));
}

template <int P>
__device__ __forceinline__ val_t<P> weight(const QuadW &w, int q) {
    if constexpr (P == FEM_FP64) return w.wd[q];
    else return w.wf[q];
}

template <int DIM, int P, int CPT, bool ADJ>
__global__ void __launch_bounds__(kBlock) lap_kernel(const __grid_constant__ LapArgs a) {
    constexpr int NB = DIM + 1;
    using T = val_t<P>;
    const int64_t C = a.C;
    const T *__restrict__ u = static_cast<const T *>(a.u);
    const T *__restrict__ K = static_cast<const T *>(a.K);
    T *__restrict__ out = static_cast<T *>(a.out);
    const double *X[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) X[k] = a.X[k];

    const int64_t ngroups = (C + CPT - 1) / CPT;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < ngroups; g += stride) {
        const int64_t c0 = g * CPT;
        int32_t vid[NB][CPT];
#pragma unroll
        for (int b = 0; b < NB; ++b) load_row<CPT>(a.conn + b * C + c0, vid[b]);

        // quadrature sum of the coefficient: Kbar = sum_q w_q K_q
        qsum_t<P> ks[CPT];
        {
            T kq[CPT];
            load_row<CPT>(K + c0, kq);
#pragma unroll
            for (int i = 0; i < CPT; ++i) ks[i].first(weight<P>(a.w, 0), kq[i]);
        }
        for (int q = 1; q < a.w.nq; ++q) {
            T kq[CPT];
            load_row<CPT>(K + q * C + c0, kq);
            const T wq = weight<P>(a.w, q);
#pragma unroll
            for (int i = 0; i < CPT; ++i) ks[i].add(wq, kq[i]);
        }

        T lamv[ADJ ? NB : 1][CPT];
        if constexpr (ADJ) {
#pragma unroll
            for (int b = 0; b < NB; ++b) load_row<CPT>(static_cast<const T *>(a.lam) + b * C + c0, lamv[b]);
        }

        T r[NB][CPT];
        T tfac[CPT];
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            uint32_t v[NB];
            T uu[NB], ll[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                v[b] = clamp_vid(vid[b][i], a.V);
                uu[b] = ld_gather(u + v[b]);
                if constexpr (ADJ) ll[b] = lamv[b][i];
            }
            T rr[NB];
            T tf = T(0);
            if constexpr (P == FEM_FP64) {
                double e[DIM][DIM], n[DIM][DIM];
                columns_f64<DIM>(X, v, e);
                double det = adjugate_rows<DIM>(e, n);
                if constexpr (ADJ) {
                    lap_element<DIM>(n, det, ll, ks[i].value(), rr);
                    tf = lap_dk_factor<DIM>(n, det, uu, ll);
                } else {
                    lap_element<DIM>(n, det, uu, ks[i].value(), rr);
                }
            } else {
                float e[DIM][DIM], n[DIM][DIM];
                if constexpr (P == FEM_FP32_MIXED) columns_mixed<DIM>(X, v, e);
                else columns_f32<DIM>(X, v, e);
                float det = adjugate_rows<DIM>(e, n);
                bool ok = true;
                if constexpr (P == FEM_FP32_MIXED) ok = shape_ok<DIM>(e, det, a.tau2);
                if (ok) {
                    if constexpr (ADJ) {
                        lap_element<DIM>(n, det, ll, ks[i].value(), rr);
                        tf = lap_dk_factor<DIM>(n, det, uu, ll);
                    } else {
                        lap_element<DIM>(n, det, uu, ks[i].value(), rr);
                    }
                } else {
                    // badly shaped (or under/overflowing) cell: float64 geometry and sums
                    double e64[DIM][DIM], n64[DIM][DIM], u64[NB], r64[NB];
                    columns_f64<DIM>(X, v, e64);
                    double det64 = adjugate_rows<DIM>(e64, n64);
                    const double kb64 = ks[i].value_f64();
                    if constexpr (ADJ) {
                        double l64[NB];
#pragma unroll
                        for (int b = 0; b < NB; ++b) u64[b] = uu[b], l64[b] = ll[b];
                        lap_element<DIM>(n64, det64, l64, kb64, r64);
                        tf = static_cast<float>(lap_dk_factor<DIM>(n64, det64, u64, l64));
                    } else {
#pragma unroll
                        for (int b = 0; b < NB; ++b) u64[b] = uu[b];
                        lap_element<DIM>(n64, det64, u64, kb64, r64);
                    }
#pragma unroll
                    for (int b = 0; b < NB; ++b) rr[b] = static_cast<float>(r64[b]);
                }
            }
#pragma unroll
            for (int b = 0; b < NB; ++b) r[b][i] = rr[b];
            tfac[i] = tf;
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) store_row<CPT>(out + b * C + c0, r[b]);
        if constexpr (ADJ) {
            T *dK = static_cast<T *>(a.dK);
            for (int q = 0; q < a.w.nq; ++q) {
                const T wq = weight<P>(a.w, q);
                T row[CPT];
#pragma unroll
                for (int i = 0; i < CPT; ++i) row[i] = wq * tfac[i];
                store_row<CPT>(dK + q * C + c0, row);
            }
        }
    }
}

template <int DIM, int P, bool ADJ>
static fem_status launch_lap(const LapArgs &a, bool vec, cudaStream_t s) {
    if (vec) {
        auto k = lap_kernel<DIM, P, 4, ADJ>;
        int grid = grid_for((a.C + 3) / 4, kBlock, reinterpret_cast<const void *>(k));
        k<<<grid, kBlock, 0, s>>>(a);
    } else {
        auto k = lap_kernel<DIM, P, 1, ADJ>;
        int grid = grid_for(a.C, kBlock, reinterpret_cast<const void *>(k));
        k<<<grid, kBlock, 0, s>>>(a);
    }
    return check_launch(ADJ ? "fem_adjoint_laplacian" : "fem_integrate_laplacian");
}

template <bool ADJ>
static fem_status dispatch_lap(int dim, fem_precision prec, const LapArgs &a, bool vec, cudaStream_t s) {
    if (dim == 2) {
        switch (prec) {
            case FEM_FP64: return launch_lap<2, FEM_FP64, ADJ>(a, vec, s);
            case FEM_FP32_MIXED: return launch_lap<2, FEM_FP32_MIXED, ADJ>(a, vec, s);
            case FEM_FP32: return launch_lap<2, FEM_FP32, ADJ>(a, vec, s);
        }
    } else {
        switch (prec) {
            case FEM_FP64: return launch_lap<3, FEM_FP64, ADJ>(a, vec, s);
            case FEM_FP32_MIXED: return launch_lap<3, FEM_FP32_MIXED, ADJ>(a, vec, s);
            case FEM_FP32: return launch_lap<3, FEM_FP32, ADJ>(a, vec, s);
        }
    }
    return fail(FEM_ERR_ARG, "unknown precision %d", static_cast<int>(prec));
}

static fem_status fill_args(LapArgs &a, int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                            const int32_t *conn, const void *u, const void *K, int n_q, const double *qpts,
                            const double *qw, fem_precision prec) {
    fem_status st = check_common(dim, n_cells, n_verts, coords, conn);
    if (st != FEM_OK) return st;
    if (prec != FEM_FP64 && prec != FEM_FP32_MIXED && prec != FEM_FP32)
        return fail(FEM_ERR_ARG, "unknown precision %d", static_cast<int>(prec));
    if ((st = load_quadrature(dim, n_q, qpts, qw, a.w)) != FEM_OK) return st;
    for (int k = 0; k < 3; ++k) a.X[k] = coords + (k < dim ? k : 0) * n_verts;
    a.conn = conn;
    a.u = u;
    a.K = K;
    a.lam = nullptr;
    a.out = nullptr;
    a.dK = nullptr;
    a.C = n_cells;
    a.V = static_cast<uint32_t>(n_verts);
    float tau = mixed_tau();
    a.tau2 = tau * tau;
    return FEM_OK;
}

}  // namespace fem

using namespace fem;

extern "C" fem_status fem_integrate_laplacian(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                              const int32_t *conn, const void *u, const void *K, int n_q,
                                              const double *qpts, const double *qw, void *elem_out,
                                              fem_precision prec, fem_stream stream) {
    LapArgs a;
    fem_status st = fill_args(a, dim, n_cells, n_verts, coords, conn, u, K, n_q, qpts, qw, prec);
    if (st != FEM_OK) return st;
    if (n_cells == 0) return FEM_OK;
    if (!u || !K || !elem_out) return fail(FEM_ERR_ARG, "u, K or elem_out is NULL");
    a.out = elem_out;
    const bool vec = n_cells % 4 == 0 && aligned16(conn) && aligned16(K) && aligned16(elem_out);
    return dispatch_lap<false>(dim, prec, a, vec, stream);
}

namespace fem {
fem_status launch_gather(int dim, int n_comp, int64_t C, int64_t V, const void *elem, const int32_t *node_ptr,
                         const int32_t *node_idx, void *out, fem_precision prec, cudaStream_t s);
}

extern "C" fem_status fem_adjoint_laplacian(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                            const int32_t *conn, const void *u, const void *K, int n_q,
                                            const double *qpts, const double *qw, const void *lambda, void *dK,
                                            void *du, const int32_t *node_ptr, const int32_t *node_idx,
                                            void *scratch, fem_precision prec, fem_stream stream) {
    LapArgs a;
    fem_status st = fill_args(a, dim, n_cells, n_verts, coords, conn, u, K, n_q, qpts, qw, prec);
    if (st != FEM_OK) return st;
    if (n_verts > 0 && (!du || !node_ptr)) return fail(FEM_ERR_ARG, "du or node_ptr is NULL");
    if (n_cells > 0 && (!u || !K || !lambda || !dK || !node_idx || !scratch))
        return fail(FEM_ERR_ARG, "a NULL adjoint argument");
    if (n_cells > 0) {
        a.lam = lambda;
        a.out = scratch;
        a.dK = dK;
        const bool vec = n_cells % 4 == 0 && aligned16(conn) && aligned16(K) && aligned16(lambda) &&
                         aligned16(dK) && aligned16(scratch);
        if ((st = dispatch_lap<true>(dim, prec, a, vec, stream)) != FEM_OK) return st;
    }
    return launch_gather(dim, 1, n_cells, n_verts, scratch, node_ptr, node_idx, du, prec, stream);
}
