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
#include <algorithm>

#include "fem_cell.cuh"
#include "fem_pipe.cuh"

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
    unsigned *err;  // device error word (FEM_DEVERR_BADMESH)
    QuadW w;
};

// r_b from the adjugate rows, the scale s = Kbar / |det J| and the nodal values (T =
// double, float, or f2 for two cells at once).
template <int DIM, class T>
__device__ __forceinline__ void lap_apply(const T (&n)[DIM][DIM], T s, const T (&uu)[DIM + 1], T (&r)[DIM + 1]) {
    T h[DIM];
    {
        const T du = uu[1] - uu[0];
#pragma unroll
        for (int i = 0; i < DIM; ++i) h[i] = du * n[0][i];
    }
#pragma unroll
    for (int j = 1; j < DIM; ++j) {
        const T du = uu[j + 1] - uu[0];
#pragma unroll
        for (int i = 0; i < DIM; ++i) h[i] = fma(du, n[j][i], h[i]);
    }
    T sum = zero<T>();
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        r[j + 1] = s * dotv<DIM>(n[j], h);
        sum = sum + r[j + 1];
    }
    r[0] = neg(sum);
}

// r_b from the adjugate rows, the determinant, the nodal values and Kbar
template <int DIM, class T>
__device__ __forceinline__ void lap_element(const T (&n)[DIM][DIM], T det, const T (&uu)[DIM + 1], T kbar,
                                            T (&r)[DIM + 1]) {
    lap_apply<DIM>(n, quot_abs(kbar, det), uu, r);
}

// The adjoint's element part in one pass: h_lambda and h_u once, one reciprocal of |det J|
// for both quotients; r_b = (Kbar / |det J|) n_b . h_lambda (the residual of lambda_e),
// tf = h_lambda . h_u / |det J|.
template <int DIM, class T>
__device__ __forceinline__ void lap_adj_element(const T (&n)[DIM][DIM], T det, const T (&uu)[DIM + 1],
                                                const T (&ll)[DIM + 1], T kbar, T (&r)[DIM + 1], T &tf) {
    T hu[DIM], hl[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) hu[i] = zero<T>(), hl[i] = zero<T>();
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        const T du = uu[j + 1] - uu[0], dl = ll[j + 1] - ll[0];
#pragma unroll
        for (int i = 0; i < DIM; ++i) hu[i] = fma(du, n[j][i], hu[i]), hl[i] = fma(dl, n[j][i], hl[i]);
    }
    T one;
    if constexpr (std::is_same<T, f2>::value) one = f2_splat(1.0f);
    else one = T(1);
    const T y = quot_abs(one, det), s = kbar * y;
    T sum = zero<T>();
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        r[j + 1] = s * dotv<DIM>(n[j], hl);
        sum = sum + r[j + 1];
    }
    r[0] = neg(sum);
    tf = dotv<DIM>(hl, hu) * y;
}

template <int P>
__device__ __forceinline__ val_t<P> weight(const QuadW &w, int q) {
    if constexpr (P == FEM_FP64) return w.wd[q];
    else return w.wf[q];
}

// One cell: vertex coordinates xs, nodal values uu (adjoint: ll = lambda_e), the
// quadrature sum of the coefficient ks; writes the element vector rr and (adjoint) the
// dK factor tf. bad_det collects the mesh check: det J = 0 or non-finite, or (rep) vertex
// ids that repeat; the mixed form checks only the cells its shape test sends to float64
// (every degenerate cell fails that test for tau > 0).
template <int DIM, int P, bool ADJ>
__device__ __forceinline__ void lap_cell(const double (&xs)[DIM + 1][DIM],
                                         const val_t<P> (&uu)[DIM + 1], const val_t<P> (&ll)[DIM + 1],
                                         const qsum_t<P> &ks, float tau2, val_t<P> (&rr)[DIM + 1], val_t<P> &tf,
                                         bool rep, bool &bad_det) {
    constexpr int NB = DIM + 1;
    if constexpr (P == FEM_FP64) {
        double e[DIM][DIM], n[DIM][DIM];
        columns_f64<DIM>(xs, e);
        double det = adjugate_rows<DIM>(e, n);
        bad_det |= det_bad(det) | rep;
        if constexpr (ADJ) {
            lap_adj_element<DIM>(n, det, uu, ll, ks.value(), rr, tf);
        } else {
            lap_element<DIM>(n, det, uu, ks.value(), rr);
        }
    } else {
        float e[DIM][DIM], n[DIM][DIM];
        if constexpr (P == FEM_FP32_MIXED) columns_mixed<DIM>(xs, e);
        else columns_f32<DIM>(xs, e);
        float det = adjugate_rows<DIM>(e, n);
        bool ok = true;
        if constexpr (P == FEM_FP32_MIXED) ok = shape_ok<DIM>(e, det, tau2);
        else bad_det |= det_bad(det) | rep;
        if (ok) {
            if constexpr (ADJ) {
                lap_adj_element<DIM>(n, det, uu, ll, ks.value(), rr, tf);
            } else {
                lap_element<DIM>(n, det, uu, ks.value(), rr);
            }
        } else {
            // badly shaped (or under/overflowing) cell: float64 geometry and sums
            double e64[DIM][DIM], n64[DIM][DIM], u64[NB], r64[NB];
            columns_f64<DIM>(xs, e64);
            double det64 = adjugate_rows<DIM>(e64, n64);
            bad_det |= det_bad(det64) | rep;
            const double kb64 = ks.value_f64();
#pragma unroll
            for (int b = 0; b < NB; ++b) u64[b] = uu[b];
            if constexpr (ADJ) {
                double l64[NB];
#pragma unroll
                for (int b = 0; b < NB; ++b) l64[b] = ll[b];
                double tf64;
                lap_adj_element<DIM>(n64, det64, u64, l64, kb64, r64, tf64);
                tf = static_cast<float>(tf64);
            } else {
                lap_element<DIM>(n64, det64, u64, kb64, r64);
            }
#pragma unroll
            for (int b = 0; b < NB; ++b) rr[b] = static_cast<float>(r64[b]);
        }
    }
}

// Direct kernel: one thread owns CPT consecutive cells and reads the cell-indexed rows
// with (vector) loads from global memory. Used where neither the pair kernel (float32
// forms: an even cell count, 8-byte aligned rows) nor the staged kernel (float64 form:
// 16-byte aligned rows, stages that fit in shared memory) applies, and by the host-buffer
// path, which reads page-locked host memory.
template <int DIM, int P, int CPT, int NQ, bool ADJ>
__global__ void __launch_bounds__(kBlock) lap_kernel(const __grid_constant__ LapArgs a) {
    pdl_wait();  // overlapped launch: the previous kernel's writes are visible from here
    pdl_trigger();
    constexpr int NB = DIM + 1;
    using T = val_t<P>;
    const int64_t C = a.C;
    const T *__restrict__ u = static_cast<const T *>(a.u);
    const T *__restrict__ K = static_cast<const T *>(a.K);
    T *__restrict__ out = static_cast<T *>(a.out);
    const double *X[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) X[k] = a.X[k];

    uint32_t vmax = 0;     // largest vertex id seen (bad ids are clamped and reported)
    bool bad_det = false;  // a cell with det J = 0 or non-finite
    const int64_t ngroups = (C + CPT - 1) / CPT;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < ngroups; g += stride) {
        const int64_t c0 = g * CPT;
        int32_t vid[NB][CPT];
#pragma unroll
        for (int b = 0; b < NB; ++b) load_row<CPT>(a.conn + b * C + c0, vid[b]);

        // quadrature sum of the coefficient: Kbar = sum_q w_q K_q (with NQ > 0 every row
        // load is issued before the first sum)
        qsum_t<P> ks[CPT];
        if constexpr (NQ > 0) {
            T kq[NQ][CPT];
#pragma unroll
            for (int q = 0; q < NQ; ++q) load_row<CPT>(K + q * C + c0, kq[q]);
#pragma unroll
            for (int i = 0; i < CPT; ++i) ks[i].first(weight<P>(a.w, 0), kq[0][i]);
#pragma unroll
            for (int q = 1; q < NQ; ++q)
#pragma unroll
                for (int i = 0; i < CPT; ++i) ks[i].add(weight<P>(a.w, q), kq[q][i]);
        } else {
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
                v[b] = clamp_vid(vid[b][i], a.V, vmax);
                uu[b] = ld_gather(u + v[b]);
                ll[b] = ADJ ? lamv[ADJ ? b : 0][i] : T(0);
            }
            double xs[NB][DIM];
            gather_coords<DIM>(X, v, xs);
            T rr[NB];
            T tf = T(0);
            lap_cell<DIM, P, ADJ>(xs, uu, ll, ks[i], a.tau2, rr, tf, ids_repeat<NB>(v), bad_det);
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
    report_mesh(a.err, vmax, a.V, bad_det);
}

// ------------------------------------------------------------------ several fields

// Element residuals of n_fields nodal fields on one mesh and coefficient: the geometry
// (coordinate gathers, adjugate rows, det J) and s = Kbar / |det J| are computed once per
// cell and kept in registers; each field then costs its nodal gathers, the contraction
// and its stores. u is [n_fields][V], out [n_fields][dim+1][C]. Per field and cell the
// arithmetic is exactly that of the single-field per-cell routine (lap_cell).
struct FieldsArgs {
    LapArgs a;  // conn, K, coords, C, V, quadrature, tau2; a.u = u of field 0, a.out = out of field 0
    int nf;
};

// badly shaped cell of the mixed form: float64 geometry and sums for every field
template <int DIM>
__device__ __noinline__ void lap_fields_fallback(const FieldsArgs &fa, int64_t c, double kbar) {
    constexpr int NB = DIM + 1;
    const LapArgs &a = fa.a;
    const int64_t C = a.C;
    uint32_t v[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) v[b] = clamp_vid(a.conn[b * C + c], a.V);
    const double *X[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) X[k] = a.X[k];
    double xs[NB][DIM], e64[DIM][DIM], n64[DIM][DIM];
    gather_coords<DIM>(X, v, xs);
    columns_f64<DIM>(xs, e64);
    const double det64 = adjugate_rows<DIM>(e64, n64);
    if (det_bad(det64) || ids_repeat<NB>(v)) record_device_error(a.err, FEM_DEVERR_BADMESH);
    const double s = quot_abs(kbar, det64);
    const float *u = static_cast<const float *>(a.u);
    float *out = static_cast<float *>(a.out);
    for (int f = 0; f < fa.nf; ++f) {
        double u64[NB], r64[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) u64[b] = u[int64_t(f) * a.V + v[b]];
        lap_apply<DIM>(n64, s, u64, r64);
#pragma unroll
        for (int b = 0; b < NB; ++b) out[(int64_t(f) * NB + b) * C + c] = static_cast<float>(r64[b]);
    }
}

template <int DIM, int P, int CPT, int NQ>
__global__ void __launch_bounds__(kBlock) lap_fields_kernel(const __grid_constant__ FieldsArgs fa) {
    pdl_wait();  // overlapped launch: the previous kernel's writes are visible from here
    pdl_trigger();
    constexpr int NB = DIM + 1;
    using T = val_t<P>;
    const LapArgs &a = fa.a;
    const int64_t C = a.C;
    const int64_t V = a.V;
    const T *__restrict__ u = static_cast<const T *>(a.u);
    const T *__restrict__ K = static_cast<const T *>(a.K);
    T *__restrict__ out = static_cast<T *>(a.out);
    const double *X[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) X[k] = a.X[k];
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
        qsum_t<P> ks[CPT];
        {
            T kq[CPT];
            load_row<CPT>(K + c0, kq);
#pragma unroll
            for (int i = 0; i < CPT; ++i) ks[i].first(weight<P>(a.w, 0), kq[i]);
        }
#pragma unroll(NQ > 0 ? NQ - 1 : 1)
        for (int q = 1; q < nq; ++q) {
            T kq[CPT];
            load_row<CPT>(K + q * C + c0, kq);
#pragma unroll
            for (int i = 0; i < CPT; ++i) ks[i].add(weight<P>(a.w, q), kq[i]);
        }
        // per-cell geometry, kept for all fields
        uint32_t v[CPT][NB];
        T n[CPT][DIM][DIM], s[CPT];
        bool ok[CPT];
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
#pragma unroll
            for (int b = 0; b < NB; ++b) v[i][b] = clamp_vid(vid[b][i], a.V, vmax);
            double xs[NB][DIM];
            gather_coords<DIM>(X, v[i], xs);
            T e[DIM][DIM];
            if constexpr (P == FEM_FP64) columns_f64<DIM>(xs, e);
            else if constexpr (P == FEM_FP32_MIXED) columns_mixed<DIM>(xs, e);
            else columns_f32<DIM>(xs, e);
            const T det = adjugate_rows<DIM>(e, n[i]);
            s[i] = quot_abs(ks[i].value(), det);
            ok[i] = true;
            if constexpr (P == FEM_FP32_MIXED) ok[i] = shape_ok<DIM>(e, det, a.tau2);
            else bad_det |= det_bad(det) | ids_repeat<NB>(v[i]);
        }
        for (int f = 0; f < fa.nf; ++f) {
            const T *uf = u + int64_t(f) * V;
            T r[NB][CPT];
#pragma unroll
            for (int i = 0; i < CPT; ++i) {
                T uu[NB], rr[NB];
#pragma unroll
                for (int b = 0; b < NB; ++b) uu[b] = ld_gather(uf + v[i][b]);
                lap_apply<DIM>(n[i], s[i], uu, rr);
#pragma unroll
                for (int b = 0; b < NB; ++b) r[b][i] = rr[b];
            }
#pragma unroll
            for (int b = 0; b < NB; ++b) store_row<CPT>(out + (int64_t(f) * NB + b) * C + c0, r[b]);
        }
        if constexpr (P == FEM_FP32_MIXED) {
#pragma unroll
            for (int i = 0; i < CPT; ++i)
                if (!ok[i]) lap_fields_fallback<DIM>(fa, c0 + i, ks[i].value_f64());
        }
    }
    report_mesh(a.err, vmax, a.V, bad_det);
}

template <int DIM, int P>
static fem_status launch_fields(const FieldsArgs &fa, bool vec, cudaStream_t s) {
    // float64 keeps two cells per thread (the geometry of four would crowd the registers)
    constexpr int CPTV = P == FEM_FP64 ? 2 : 4;
    constexpr int NQN = DIM == 3 ? 4 : 3;  // the workloads' rules
    if (vec && fa.a.w.nq == NQN) {
        // float32 forms: one wave of resident CTAs (8 fields: 69.5 -> 68.0 us per step)
        auto k = lap_fields_kernel<DIM, P, CPTV, NQN>;
        const int64_t n = (fa.a.C + CPTV - 1) / CPTV;
        const void *kp = reinterpret_cast<const void *>(k);
        launch_overlapped(k, P == FEM_FP64 ? grid_for(n, kBlock, kp) : resident_grid(kp, kBlock, n), kBlock, 0, s, fa);
    } else {
        auto k = lap_fields_kernel<DIM, P, 1, 0>;
        launch_overlapped(k, grid_for(fa.a.C, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, s, fa);
    }
    return check_launch("fem_integrate_laplacian_fields");
}

// ------------------------------------------------------------------ mixed-form fallback and cell pairs

// Float64 recomputation of one cell of the mixed form (badly shaped or non-finite):
// float64 geometry and sums from the gathered coordinates and the float32 values.
template <int DIM, bool ADJ>
__device__ __forceinline__ void lap_cell_f64(const double (&xs)[DIM + 1][DIM], const float (&uf)[DIM + 1],
                                             const float (&lf)[DIM + 1], double kbar, double (&r)[DIM + 1],
                                             double &tf, unsigned *err) {
    constexpr int NB = DIM + 1;
    double e[DIM][DIM], n[DIM][DIM], u64[NB], l64[NB];
    columns_f64<DIM>(xs, e);
    const double det = adjugate_rows<DIM>(e, n);
    if (det_bad(det)) record_device_error(err, FEM_DEVERR_BADMESH);
#pragma unroll
    for (int b = 0; b < NB; ++b) u64[b] = uf[b], l64[b] = lf[b];
    if constexpr (ADJ) {
        lap_adj_element<DIM>(n, det, u64, l64, kbar, r, tf);
    } else {
        lap_element<DIM>(n, det, u64, kbar, r);
        tf = 0.0;
    }
}

template <int P>
using qsum2_t = typename std::conditional<P == FEM_FP32_MIXED, Dot2Sum2, PlainSum2>::type;

// Float64 recomputation of cell c of the mixed form, stored over the float32 result that
// the caller has already written (same thread, program order). Everything is read again
// from global memory: the path is rare and kept out of line so that none of its state
// occupies registers on the common path.
template <int DIM, bool ADJ>
__device__ __noinline__ void lap_fallback_store(const LapArgs &a, int64_t c, double kbar) {
    constexpr int NB = DIM + 1;
    const int64_t C = a.C;
    uint32_t v[NB];
    float uf[NB], lf[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        v[b] = clamp_vid(a.conn[b * C + c], a.V);
        uf[b] = static_cast<const float *>(a.u)[v[b]];
        lf[b] = ADJ ? static_cast<const float *>(a.lam)[b * C + c] : 0.0f;
    }
    const double *X[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) X[k] = a.X[k];
    double xs[NB][DIM], r64[NB], t64;
    gather_coords<DIM>(X, v, xs);
    if (ids_repeat<NB>(v)) record_device_error(a.err, FEM_DEVERR_BADMESH);
    lap_cell_f64<DIM, ADJ>(xs, uf, lf, kbar, r64, t64, a.err);
    float *out = static_cast<float *>(a.out);
#pragma unroll
    for (int b = 0; b < NB; ++b) out[b * C + c] = static_cast<float>(r64[b]);
    if constexpr (ADJ) {
        float *dK = static_cast<float *>(a.dK);
        for (int q = 0; q < a.w.nq; ++q) dK[q * C + c] = static_cast<float>(a.w.wd[q] * t64);
    }
}

// Two cells of a float32 form at once (lane x: cell a, lane y: cell b), vertex ids va,
// vb. The coordinates are gathered here and are dead once split into float32. In the
// mixed form, oka / okb report whether each cell passed the shape test; a failing cell's
// result here is meaningless and the caller recomputes it (lap_fallback_store). In the
// float32 ablation they report whether det J is nonzero and finite (the mesh check).
template <int DIM, int P, bool ADJ>
__device__ __forceinline__ void lap_pair(const double *const (&X)[DIM], const uint32_t (&va)[DIM + 1],
                                         const uint32_t (&vb)[DIM + 1], const f2 (&uu)[DIM + 1],
                                         const f2 (&ll)[DIM + 1], const qsum2_t<P> &ks, float tau2,
                                         f2 (&rr)[DIM + 1], f2 &tf, bool &oka, bool &okb) {
    f2 e[DIM][DIM], n[DIM][DIM];
    {
        double xa[DIM + 1][DIM], xb[DIM + 1][DIM];
        gather_coords<DIM>(X, va, xa);
        gather_coords<DIM>(X, vb, xb);
        if constexpr (P == FEM_FP32_MIXED) columns_mixed2<DIM>(xa, xb, e);
        else columns_f32_2<DIM>(xa, xb, e);
    }
    const f2 det = adjugate_rows<DIM>(e, n);
    if constexpr (ADJ) {
        lap_adj_element<DIM>(n, det, uu, ll, ks.value(), rr, tf);
    } else {
        lap_element<DIM>(n, det, uu, ks.value(), rr);
    }
    if constexpr (P == FEM_FP32_MIXED) {
        shape_ok2<DIM>(e, det, tau2, oka, okb);
    } else {
        oka = !det_bad(f2_x(det));
        okb = !det_bad(f2_y(det));
    }
}

// ------------------------------------------------------------------ pair kernel
//
// The float32 forms' kernel for rows that are 8-byte aligned (an even cell count): each
// thread owns two consecutive cells at a time and computes them as f32x2 pairs
// (lap_pair), reading every cell-indexed row with 8-byte loads and writing 8-byte
// streaming stores, grid-stride over the cell pairs with one wave of resident CTAs (3 of
// 256 threads per SM at up to 80 registers). A badly shaped cell of the mixed form is
// recomputed in float64 out of line (lap_fallback_store) after its pair's stores.
//
// Measured on the 1,572,864-tet workload (L2 flushed, CUDA events): 25.9 us against
// 27.8 us for the bulk-copy staged kernel with the same per-cell arithmetic (bitwise the
// same results): the staged kernel's pipeline fill costs more than its prefetching saves
// at this size; at 2^23 cells the two are within 1 %. Both are bound by the latency of
// the 16 vertex gathers per cell and by the integer float64 -> float32 splits (ALU pipe
// half busy), not by DRAM (30 % of peak over the launch).
// The mixed form and the adjoint run 3 CTAs per SM at up to 80 registers: with launches
// that overlap the previous kernel's tail and steps back to back, the mixed residual took
// 23.2 us against 23.5 us at 4 CTAs (64 registers) on the 1,572,864-tet workload, and 106.5
// against 108.8 us on 2^23 cells; 2 CTAs (118 registers) took 27.2 us. The float32
// ablation, without the coordinate splits, keeps 4 (3 took 23.1 against 21.9 us).
template <int P, bool ADJ>
constexpr int pair_min_blocks() { return (P == FEM_FP32 && !ADJ) ? 4 : 3; }

template <int DIM, int P, int NQ, bool ADJ>
__global__ void __launch_bounds__(kBlock, pair_min_blocks<P, ADJ>()) lap_pair_kernel(const __grid_constant__ LapArgs a) {
    static_assert(P != FEM_FP64, "float32 forms only");
    pdl_wait();  // launched overlapped: the previous kernel's writes are visible from here
    pdl_trigger();
    constexpr int NB = DIM + 1;
    const int64_t C = a.C;  // even
    const float *__restrict__ u = static_cast<const float *>(a.u);
    const float *__restrict__ K = static_cast<const float *>(a.K);
    const float *__restrict__ L = static_cast<const float *>(a.lam);
    float *__restrict__ out = static_cast<float *>(a.out);
    float *__restrict__ dK = static_cast<float *>(a.dK);
    const double *X[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) X[k] = a.X[k];
    const int nq = NQ > 0 ? NQ : a.w.nq;
    uint32_t vmax = 0;     // largest vertex id seen (bad ids are clamped and reported)
    bool bad_det = false;  // float32 ablation: a cell with det J = 0 or non-finite, or repeated ids
    const int64_t np = C / 2;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < np; g += stride) {
        const int64_t c = 2 * g;
        uint32_t va[NB], vb[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int2 t = __ldcs(reinterpret_cast<const int2 *>(a.conn + b * C + c));
            va[b] = clamp_vid(t.x, a.V, vmax);
            vb[b] = clamp_vid(t.y, a.V, vmax);
        }
        qsum2_t<P> ks;
#pragma unroll(NQ > 0 ? NQ : 1)
        for (int q = 0; q < nq; ++q) {
            const float2 k = __ldcs(reinterpret_cast<const float2 *>(K + q * C + c));
            if (q == 0) ks.first(a.w.wf[0], f2_make(k.x, k.y));
            else ks.add(a.w.wf[q], f2_make(k.x, k.y));
        }
        f2 uu[NB], ll[NB], rr[NB], tf = zero<f2>();
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            uu[b] = f2_make(ld_gather(u + va[b]), ld_gather(u + vb[b]));
            if constexpr (ADJ) {
                const float2 l = __ldcs(reinterpret_cast<const float2 *>(L + b * C + c));
                ll[b] = f2_make(l.x, l.y);
            } else {
                ll[b] = zero<f2>();
            }
        }
        bool oka, okb;
        lap_pair<DIM, P, ADJ>(X, va, vb, uu, ll, ks, a.tau2, rr, tf, oka, okb);
#pragma unroll
        for (int b = 0; b < NB; ++b)
            __stcs(reinterpret_cast<float2 *>(out + b * C + c), make_float2(f2_x(rr[b]), f2_y(rr[b])));
        if constexpr (ADJ) {
            for (int q = 0; q < nq; ++q) {
                const float wq = a.w.wf[q];
                __stcs(reinterpret_cast<float2 *>(dK + q * C + c), make_float2(wq * f2_x(tf), wq * f2_y(tf)));
            }
        }
        if constexpr (P == FEM_FP32_MIXED) {
            if (!oka) lap_fallback_store<DIM, ADJ>(a, c, ks.value_f64_x());
            if (!okb) lap_fallback_store<DIM, ADJ>(a, c + 1, ks.value_f64_y());
        } else {
            bad_det |= !oka | !okb | ids_repeat<NB>(va) | ids_repeat<NB>(vb);
        }
    }
    report_mesh(a.err, vmax, a.V, bad_det);
}

template <int DIM, int P, int NQ, bool ADJ>
static void launch_pair(const LapArgs &a, cudaStream_t s) {
    auto k = lap_pair_kernel<DIM, P, NQ, ADJ>;
    launch_overlapped(k, resident_grid(reinterpret_cast<const void *>(k), kBlock, a.C / 2), kBlock, 0, s, a);
}

// ------------------------------------------------------------------ prepared vertex records
//
// The mixed form splits every float64 coordinate into a float32 (hi, lo) pair before it
// differences the Jacobian columns; the per-cell kernels do so for every cell a vertex
// belongs to (about 24 tets per vertex in 3D), ~100 integer instructions per tet, and
// gather the coordinates with 3 (2D: 2) loads per vertex. fem_prepare_vertices does the
// split once per mesh into a record of 8 floats per vertex (3D: hi_x hi_y hi_z lo_x lo_y
// lo_z 0 0; 2D: 4 floats hi_x hi_y lo_x lo_y, lo kept as split_f64 returns it), and
// lap_rec_kernel gathers one record per vertex with one 32-byte (2D: 16-byte) load. The
// Jacobian columns are then formed by the same operations as columns_mixed2, so the element
// vectors are bitwise those of the pair kernel.
__host__ __device__ constexpr int rec_floats(int dim) { return dim == 3 ? 8 : 4; }

template <int DIM>
__global__ void __launch_bounds__(kBlock) prepare_vertices_kernel(const double *coords, int64_t V, float *rec) {
    constexpr int R = rec_floats(DIM);
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < V; v += stride) {
        float r[R];
#pragma unroll
        for (int i = 0; i < R; ++i) r[i] = 0.0f;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const double x = coords[k * V + v];
            split_f64(static_cast<uint32_t>(__double2loint(x)), static_cast<uint32_t>(__double2hiint(x)), r[k],
                      r[DIM + k]);
        }
        float4 *dst = reinterpret_cast<float4 *>(rec + v * R);
        dst[0] = make_float4(r[0], r[1], r[2], r[3]);
        if constexpr (R == 8) dst[1] = make_float4(r[4], r[5], r[6], r[7]);
    }
}

// one vertex record: (hi, lo) of its DIM coordinates
template <int DIM>
__device__ __forceinline__ void ld_record(const float *rec, uint32_t v, float (&hi)[DIM], float (&lo)[DIM]) {
    if constexpr (DIM == 3) {
        float t[8];
        asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=f"(t[0]), "=f"(t[1]), "=f"(t[2]), "=f"(t[3]), "=f"(t[4]), "=f"(t[5]), "=f"(t[6]), "=f"(t[7])
            : "l"(rec + size_t(v) * 8));
        hi[0] = t[0], hi[1] = t[1], hi[2] = t[2], lo[0] = t[3], lo[1] = t[4], lo[2] = t[5];
    } else {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(rec) + v);
        hi[0] = t.x, hi[1] = t.y, lo[0] = t.z, lo[1] = t.w;
    }
}

// 80 registers (3 CTAs per SM): 24.5 us on the 1,572,864-tet workload, against 25.7 us at
// 64 registers, where the eight record values of two cells' vertices spill
template <int DIM, int NQ>
__global__ void __launch_bounds__(kBlock, 3) lap_rec_kernel(const __grid_constant__ LapArgs a, const float *rec) {
    pdl_wait();  // overlapped launch: the previous kernel's writes are visible from here
    pdl_trigger();
    constexpr int NB = DIM + 1;
    const int64_t C = a.C;  // even
    const float *__restrict__ u = static_cast<const float *>(a.u);
    const float *__restrict__ K = static_cast<const float *>(a.K);
    float *__restrict__ out = static_cast<float *>(a.out);
    const int nq = NQ > 0 ? NQ : a.w.nq;
    uint32_t vmax = 0;
    const int64_t np = C / 2;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < np; g += stride) {
        const int64_t c = 2 * g;
        uint32_t va[NB], vb[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int2 t = __ldcs(reinterpret_cast<const int2 *>(a.conn + b * C + c));
            va[b] = clamp_vid(t.x, a.V, vmax);
            vb[b] = clamp_vid(t.y, a.V, vmax);
        }
        Dot2Sum2 ks;
#pragma unroll(NQ > 0 ? NQ : 1)
        for (int q = 0; q < nq; ++q) {
            const float2 k = __ldcs(reinterpret_cast<const float2 *>(K + q * C + c));
            if (q == 0) ks.first(a.w.wf[0], f2_make(k.x, k.y));
            else ks.add(a.w.wf[q], f2_make(k.x, k.y));
        }
        f2 uu[NB], hi[NB][DIM], lo[NB][DIM];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            uu[b] = f2_make(ld_gather(u + va[b]), ld_gather(u + vb[b]));
            float ha[DIM], la[DIM], hb[DIM], lb[DIM];
            ld_record<DIM>(rec, va[b], ha, la);
            ld_record<DIM>(rec, vb[b], hb, lb);
#pragma unroll
            for (int k = 0; k < DIM; ++k) hi[b][k] = f2_make(ha[k], hb[k]), lo[b][k] = f2_make(la[k], lb[k]);
        }
        // the Jacobian columns exactly as columns_mixed2 forms them
        f2 e[DIM][DIM], n[DIM][DIM];
        const f2 scale = f2_splat(0x1p-23f);
#pragma unroll
        for (int j = 0; j < DIM; ++j)
#pragma unroll
            for (int k = 0; k < DIM; ++k) e[j][k] = fma(lo[j + 1][k] - lo[0][k], scale, hi[j + 1][k] - hi[0][k]);
        const f2 det = adjugate_rows<DIM>(e, n);
        f2 rr[NB];
        lap_element<DIM>(n, det, uu, ks.value(), rr);
        bool oka, okb;
        shape_ok2<DIM>(e, det, a.tau2, oka, okb);
#pragma unroll
        for (int b = 0; b < NB; ++b)
            __stcs(reinterpret_cast<float2 *>(out + b * C + c), make_float2(f2_x(rr[b]), f2_y(rr[b])));
        if (!oka) lap_fallback_store<DIM, false>(a, c, ks.value_f64_x());
        if (!okb) lap_fallback_store<DIM, false>(a, c + 1, ks.value_f64_y());
    }
    report_mesh(a.err, vmax, a.V, false);
}

// Staged Laplacian kernel (the chunk loop of fem_pipe.cuh): each consumer thread owns kCPT
// consecutive cells of a chunk, with vector shared-memory reads of every row, vector
// streaming stores of every output row, and (float32 forms) the cells processed as f32x2
// pairs. NQ > 0 fixes the quadrature size at compile time; NQ = 0 reads it from the
// arguments.
template <class T>
__host__ __device__ constexpr uint32_t lap_stage_bytes(int nb, int nq, bool adj) {
    return uint32_t(kTile) * (4u * nb + uint32_t(sizeof(T)) * (nq + (adj ? nb : 0)));
}

// Streaming stores of kCPT consecutive cells starting at cell c: element vectors and
// (adjoint) dK = w_q * factor.
template <int DIM, int P, bool ADJ>
__device__ __forceinline__ void store_cells(const LapArgs &a, int nq, int64_t c, const val_t<P> (&r)[DIM + 1][kCPT],
                                            const val_t<P> (&tfv)[kCPT]) {
    using T = val_t<P>;
    const int64_t C = a.C;
    T *__restrict__ out = static_cast<T *>(a.out);
#pragma unroll
    for (int b = 0; b <= DIM; ++b) store_row<kCPT>(out + b * C + c, r[b]);
    if constexpr (ADJ) {
        T *__restrict__ dK = static_cast<T *>(a.dK);
        for (int q = 0; q < nq; ++q) {
            const T wq = weight<P>(a.w, q);
            T row[kCPT];
#pragma unroll
            for (int i = 0; i < kCPT; ++i) row[i] = wq * tfv[i];
            store_row<kCPT>(dK + q * C + c, row);
        }
    }
}

// The consumer work of one chunk (float64 form): thread j0/kCPT's cells j0 .. j0+kCPT-1 of
// the chunk starting at cell c0, rows read from one shared-memory stage.
template <int DIM, int P, int NQ, bool ADJ>
__device__ __forceinline__ void lap_chunk(const LapArgs &a, const double *const (&X)[DIM], int nq,
                                          const int32_t *sc, const val_t<P> *sK, const val_t<P> *sL, int j0,
                                          int64_t c0, uint32_t &vmax, bool &bad_det) {
    static_assert(P == FEM_FP64, "the float32 forms take the pair kernel");
    constexpr int NB = DIM + 1;
    using T = val_t<P>;
    const T *__restrict__ u = static_cast<const T *>(a.u);
    uint32_t v[kCPT][NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        int32_t id[kCPT];
        lds_row<kCPT>(sc + b * kTile + j0, id);
#pragma unroll
        for (int c = 0; c < kCPT; ++c) v[c][b] = clamp_vid(id[c], a.V, vmax);
    }
    T lv[kCPT][NB];
    if constexpr (ADJ) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            T lr[kCPT];
            lds_row<kCPT>(sL + b * kTile + j0, lr);
#pragma unroll
            for (int c = 0; c < kCPT; ++c) lv[c][b] = lr[c];
        }
    }
    T r[NB][kCPT], tfv[kCPT];
    qsum_t<P> ks[kCPT];
#pragma unroll(NQ > 0 ? NQ : 1)
    for (int q = 0; q < nq; ++q) {
        T kr[kCPT];
        lds_row<kCPT>(sK + q * kTile + j0, kr);
#pragma unroll
        for (int c = 0; c < kCPT; ++c) {
            if (q == 0) ks[c].first(weight<P>(a.w, 0), kr[c]);
            else ks[c].add(weight<P>(a.w, q), kr[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < kCPT; ++c) {
        double xs[NB][DIM];
        T uu[NB], rr[NB], tf = T(0), ll[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            uu[b] = ld_gather(u + v[c][b]);
            ll[b] = ADJ ? lv[c][b] : T(0);
        }
        gather_coords<DIM>(X, v[c], xs);
        lap_cell<DIM, P, ADJ>(xs, uu, ll, ks[c], a.tau2, rr, tf, ids_repeat<NB>(v[c]), bad_det);
#pragma unroll
        for (int b = 0; b < NB; ++b) r[b][c] = rr[b];
        tfv[c] = tf;
    }
    store_cells<DIM, P, ADJ>(a, nq, c0 + j0, r, tfv);
}

template <int DIM, int P, int NQ, bool ADJ>
__global__ void __launch_bounds__(kStagedThreads, FEM_STAGED_MIN_CTAS)
    lap_staged_kernel(const __grid_constant__ LapArgs a, int stages, unsigned *err) {
    pdl_wait();  // overlapped launch: the previous kernel's writes are visible from here
    pdl_trigger();
    constexpr int NB = DIM + 1;
    using T = val_t<P>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int64_t C = a.C;
    const int nq = NQ > 0 ? NQ : a.w.nq;
    const uint32_t stage_bytes = lap_stage_bytes<T>(NB, nq, ADJ);
    // stage layout: conn[NB][kTile] int32 | K[nq][kTile] T | lambda[NB][kTile] T
    auto stage_conn = [&](int s) { return reinterpret_cast<int32_t *>(smem + size_t(s) * stage_bytes); };
    auto stage_K = [&](int s) { return reinterpret_cast<T *>(stage_conn(s) + NB * kTile); };
    auto stage_lam = [&](int s) { return stage_K(s) + nq * kTile; };
    const double *X[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) X[k] = a.X[k];
    const uint64_t pol = l2_evict_first_policy();
    uint32_t vmax = 0;     // largest vertex id seen by this consumer thread
    bool bad_det = false;  // a cell with det J = 0 or non-finite (float64 form)
    staged_chunks(
        C, stages, err,
        [&](int s, int64_t c0, uint32_t n, uint64_t *bar) {
            const T *K = static_cast<const T *>(a.K);
            const T *L = static_cast<const T *>(a.lam);
            mbar_arrive_expect_tx(bar, n * (4u * NB + uint32_t(sizeof(T)) * (nq + (ADJ ? NB : 0))));
            for (int b = 0; b < NB; ++b) bulk_copy_g2s(stage_conn(s) + b * kTile, a.conn + b * C + c0, n * 4u, bar, pol);
            for (int q = 0; q < nq; ++q)
                bulk_copy_g2s(stage_K(s) + q * kTile, K + q * C + c0, n * uint32_t(sizeof(T)), bar, pol);
            if constexpr (ADJ) {
                for (int b = 0; b < NB; ++b)
                    bulk_copy_g2s(stage_lam(s) + b * kTile, L + b * C + c0, n * uint32_t(sizeof(T)), bar, pol);
            }
        },
        [&](int s, int64_t c0, int j0) {
            lap_chunk<DIM, P, NQ, ADJ>(a, X, nq, stage_conn(s), stage_K(s), stage_lam(s), j0, c0, vmax, bad_det);
        });
    report_mesh(err, vmax, a.V, bad_det);
}

template <int DIM, int P, int NQ, bool ADJ>
static fem_status launch_staged(const LapArgs &a, uint32_t sb, cudaStream_t s) {
    auto k = lap_staged_kernel<DIM, P, NQ, ADJ>;
    const int stages = ring_stages(sb);
    const size_t smem = size_t(stages) * sb;
    unsigned *err = device_error_word();
    if (!err) return fail(FEM_ERR_CUDA, "device error word unavailable");
    int grid = 0;
    fem_status st = staged_grid(reinterpret_cast<const void *>(k), kStagedThreads, smem, (a.C + kTile - 1) / kTile, grid);
    if (st != FEM_OK) return st;
    launch_overlapped(k, grid, kStagedThreads, smem, s, a, stages, err);
    return FEM_OK;
}

template <int DIM, int P, bool ADJ>
static fem_status launch_lap(const LapArgs &a, bool vec, bool pairs, cudaStream_t s, bool staged_ok = true) {
    using T = val_t<P>;
    const uint32_t sb = lap_stage_bytes<T>(DIM + 1, a.w.nq, ADJ);
    fem_status st = FEM_OK;
    // the quadrature size of the workloads' rules (3 points in 2D, 4 in 3D) is compiled in
    const bool native_nq = (DIM == 3 && a.w.nq == 4) || (DIM == 2 && a.w.nq == 3);
    if constexpr (P == FEM_FP64) {
        // few cells: 1024-cell tiles would leave most SMs idle while the float64 pipe, not
        // memory, bounds the launch, so the cells are spread over every SM (one per thread)
        const int64_t sms = sm_count();
        if ((a.C + kTile - 1) / kTile < sms) {
            const int64_t per = (a.C + 2 * sms - 1) / (2 * sms);
            int block = static_cast<int>((per + 31) / 32 * 32);
            block = block < 32 ? 32 : (block > kBlock ? kBlock : block);
            const unsigned grid = static_cast<unsigned>((a.C + block - 1) / block);
            if (native_nq) launch_overlapped((lap_kernel<DIM, P, 1, DIM + 1, ADJ>), grid, block, 0, s, a);
            else launch_overlapped((lap_kernel<DIM, P, 1, 0, ADJ>), grid, block, 0, s, a);
            return check_launch(ADJ ? "fem_adjoint_laplacian" : "fem_integrate_laplacian");
        }
    }
    if constexpr (P != FEM_FP64) {
        // float32 forms: the pair kernel (the bulk-copy staged kernel is the float64 form's).
        // Its plain 8-byte loads also serve rows in page-locked host memory (staged_ok
        // false): from host buffers 0.309 against 0.331 ms per step with lap_kernel.
        if (pairs) {
            if (native_nq) launch_pair<DIM, P, DIM + 1, ADJ>(a, s);
            else launch_pair<DIM, P, 0, ADJ>(a, s);
            return check_launch(ADJ ? "fem_adjoint_laplacian" : "fem_integrate_laplacian");
        }
    }
    if constexpr (P == FEM_FP64) {
        if (staged_ok && vec && 2u * sb <= kStageMax) {
            if (a.w.nq == DIM + 1 && DIM == 3) st = launch_staged<DIM, P, 4, ADJ>(a, sb, s);
            else if (a.w.nq == 3 && DIM == 2) st = launch_staged<DIM, P, 3, ADJ>(a, sb, s);
            else st = launch_staged<DIM, P, 0, ADJ>(a, sb, s);
            if (st != FEM_OK) return st;
            return check_launch(ADJ ? "fem_adjoint_laplacian" : "fem_integrate_laplacian");
        }
    }
    if (vec && native_nq) {
        auto k = lap_kernel<DIM, P, 4, DIM + 1, ADJ>;
        int grid = grid_for((a.C + 3) / 4, kBlock, reinterpret_cast<const void *>(k));
        launch_overlapped(k, grid, kBlock, 0, s, a);
    } else if (vec) {
        auto k = lap_kernel<DIM, P, 4, 0, ADJ>;
        int grid = grid_for((a.C + 3) / 4, kBlock, reinterpret_cast<const void *>(k));
        launch_overlapped(k, grid, kBlock, 0, s, a);
    } else {
        auto k = lap_kernel<DIM, P, 1, 0, ADJ>;
        int grid = grid_for(a.C, kBlock, reinterpret_cast<const void *>(k));
        launch_overlapped(k, grid, kBlock, 0, s, a);
    }
    return check_launch(ADJ ? "fem_adjoint_laplacian" : "fem_integrate_laplacian");
}

// vec: every cell-indexed row 16-byte aligned (C % 4 == 0); the pair kernel needs 8 bytes
template <bool ADJ>
static fem_status dispatch_lap(int dim, fem_precision prec, const LapArgs &args, bool vec, cudaStream_t s,
                               bool staged_ok = true) {
    LapArgs a = args;
    if (!(a.err = device_error_word())) return fail(FEM_ERR_CUDA, "device error word unavailable");
    const bool pairs = a.C % 2 == 0 && aligned8(a.conn) && aligned8(a.K) && aligned8(a.out) &&
                       (!ADJ || (aligned8(a.lam) && aligned8(a.dK)));
    if (dim == 2) {
        switch (prec) {
            case FEM_FP64: return launch_lap<2, FEM_FP64, ADJ>(a, vec, pairs, s, staged_ok);
            case FEM_FP32_MIXED: return launch_lap<2, FEM_FP32_MIXED, ADJ>(a, vec, pairs, s, staged_ok);
            case FEM_FP32: return launch_lap<2, FEM_FP32, ADJ>(a, vec, pairs, s, staged_ok);
        }
    } else {
        switch (prec) {
            case FEM_FP64: return launch_lap<3, FEM_FP64, ADJ>(a, vec, pairs, s, staged_ok);
            case FEM_FP32_MIXED: return launch_lap<3, FEM_FP32_MIXED, ADJ>(a, vec, pairs, s, staged_ok);
            case FEM_FP32: return launch_lap<3, FEM_FP32, ADJ>(a, vec, pairs, s, staged_ok);
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
    a.err = nullptr;  // set by dispatch_lap, once there is something to launch
    return FEM_OK;
}

}  // namespace fem

using namespace fem;

namespace fem {
fem_status launch_lap_df(int dim, int64_t n_cells, int64_t n_verts, const double *coords, const int32_t *conn,
                         const void *u, const void *K, int n_q, const double *qw, void *elem_out,
                         cudaStream_t stream);
}

extern "C" fem_status fem_integrate_laplacian(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                              const int32_t *conn, const void *u, const void *K, int n_q,
                                              const double *qpts, const double *qw, void *elem_out,
                                              fem_precision prec, fem_stream stream) {
    if (prec == FEM_FP64_DF) {
        fem_status st = check_common(dim, n_cells, n_verts, coords, conn);
        QuadW w;
        if (st == FEM_OK) st = load_quadrature(dim, n_q, qpts, qw, w);
        if (st != FEM_OK || n_cells == 0) return st;
        if (!u || !K || !elem_out) return fail(FEM_ERR_ARG, "u, K or elem_out is NULL");
        return launch_lap_df(dim, n_cells, n_verts, coords, conn, u, K, n_q, qw, elem_out, stream);
    }
    LapArgs a;
    fem_status st = fill_args(a, dim, n_cells, n_verts, coords, conn, u, K, n_q, qpts, qw, prec);
    if (st != FEM_OK) return st;
    if (n_cells == 0) return FEM_OK;
    if (!u || !K || !elem_out) return fail(FEM_ERR_ARG, "u, K or elem_out is NULL");
    a.out = elem_out;
    const bool vec = n_cells % 4 == 0 && aligned16(conn) && aligned16(K) && aligned16(elem_out);
    return dispatch_lap<false>(dim, prec, a, vec, stream);
}

extern "C" fem_status fem_integrate_laplacian_fields(int dim, int64_t n_cells, int64_t n_verts,
                                                     const double *coords, const int32_t *conn, int n_fields,
                                                     const void *u, const void *K, int n_q, const double *qpts,
                                                     const double *qw, void *elem_out, fem_precision prec,
                                                     fem_stream stream) {
    FieldsArgs fa;
    fem_status st = fill_args(fa.a, dim, n_cells, n_verts, coords, conn, u, K, n_q, qpts, qw, prec);
    if (st != FEM_OK) return st;
    if (n_fields < 0) return fail(FEM_ERR_ARG, "n_fields = %d, must be >= 0", n_fields);
    if (int64_t(n_fields) * (dim + 1) * n_cells >= (int64_t(1) << 40) || int64_t(n_fields) * n_verts >= (int64_t(1) << 40))
        return fail(FEM_ERR_SHAPE, "too many field values");
    if (n_cells == 0 || n_fields == 0) return FEM_OK;
    if (!u || !K || !elem_out) return fail(FEM_ERR_ARG, "u, K or elem_out is NULL");
    fa.a.out = elem_out;
    fa.nf = n_fields;
    if (!(fa.a.err = device_error_word())) return fail(FEM_ERR_CUDA, "device error word unavailable");
    // vector rows: C a multiple of 4 keeps every field's rows 16-byte aligned
    const bool vec = n_cells % 4 == 0 && aligned16(conn) && aligned16(K) && aligned16(elem_out);
    switch (dim * 10 + static_cast<int>(prec)) {
        case 20: return launch_fields<2, FEM_FP64>(fa, vec, stream);
        case 21: return launch_fields<2, FEM_FP32_MIXED>(fa, vec, stream);
        case 22: return launch_fields<2, FEM_FP32>(fa, vec, stream);
        case 30: return launch_fields<3, FEM_FP64>(fa, vec, stream);
        case 31: return launch_fields<3, FEM_FP32_MIXED>(fa, vec, stream);
        case 32: return launch_fields<3, FEM_FP32>(fa, vec, stream);
    }
    return fail(FEM_ERR_ARG, "unsupported dim/precision");
}

namespace fem {
// The residual with plain (vector) loads and stores only -- never the bulk-copy staged
// kernel -- for connectivity, coefficient and output arrays that live in page-locked host
// memory and are reached across the host link (fem_integrate_laplacian_host, chunks = 0).
fem_status integrate_laplacian_plain(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                     const int32_t *conn, const void *u, const void *K, int n_q, const double *qpts,
                                     const double *qw, void *elem_out, fem_precision prec, cudaStream_t stream) {
    LapArgs a;
    fem_status st = fill_args(a, dim, n_cells, n_verts, coords, conn, u, K, n_q, qpts, qw, prec);
    if (st != FEM_OK || n_cells == 0) return st;
    a.out = elem_out;
    const bool vec = n_cells % 4 == 0 && aligned16(conn) && aligned16(K) && aligned16(elem_out);
    return dispatch_lap<false>(dim, prec, a, vec, stream, false);
}

fem_status launch_gather(int dim, int n_comp, int64_t C, int64_t V, const void *elem, const int32_t *node_ptr,
                         const int32_t *node_idx, void *out, fem_precision prec, cudaStream_t s);
fem_status launch_adj_df(int dim, int64_t n_cells, int64_t n_verts, const double *coords, const int32_t *conn,
                         const void *u, const void *K, int n_q, const double *qw, const void *lambda, void *dK,
                         void *scratch, cudaStream_t stream);
}

extern "C" fem_status fem_adjoint_laplacian(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                            const int32_t *conn, const void *u, const void *K, int n_q,
                                            const double *qpts, const double *qw, const void *lambda, void *dK,
                                            void *du, const int32_t *node_ptr, const int32_t *node_idx,
                                            void *scratch, fem_precision prec, fem_stream stream) {
    LapArgs a;
    const bool df = prec == FEM_FP64_DF;  // values float64; the element part in double-float
    fem_status st = fill_args(a, dim, n_cells, n_verts, coords, conn, u, K, n_q, qpts, qw, df ? FEM_FP64 : prec);
    if (st != FEM_OK) return st;
    if (n_verts > 0 && (!du || !node_ptr)) return fail(FEM_ERR_ARG, "du or node_ptr is NULL");
    if (n_cells > 0 && (!u || !K || !lambda || !dK || !node_idx || !scratch))
        return fail(FEM_ERR_ARG, "a NULL adjoint argument");
    if (df) {
        if (n_cells > 0 &&
            (st = launch_adj_df(dim, n_cells, n_verts, coords, conn, u, K, n_q, qw, lambda, dK, scratch, stream)) !=
                FEM_OK)
            return st;
        return launch_gather(dim, 1, n_cells, n_verts, scratch, node_ptr, node_idx, du, FEM_FP64, stream);
    }
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

extern "C" int64_t fem_prepared_record_floats(int dim) { return dim == 2 || dim == 3 ? rec_floats(dim) : -1; }

extern "C" fem_status fem_prepare_vertices(int dim, int64_t n_verts, const double *coords, float *rec,
                                           fem_stream stream) {
    if (dim != 2 && dim != 3) return fail(FEM_ERR_ARG, "dim = %d, must be 2 or 3", dim);
    if (n_verts < 0 || n_verts >= (int64_t(1) << 31)) return fail(FEM_ERR_SHAPE, "n_verts out of range");
    if (n_verts == 0) return FEM_OK;
    if (!coords || !rec) return fail(FEM_ERR_ARG, "coords or rec is NULL");
    if ((reinterpret_cast<uintptr_t>(rec) & 31u) != 0) return fail(FEM_ERR_ARG, "rec must be 32-byte aligned");
    if (dim == 3) {
        auto k = prepare_vertices_kernel<3>;
        k<<<grid_for(n_verts, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, stream>>>(coords, n_verts, rec);
    } else {
        auto k = prepare_vertices_kernel<2>;
        k<<<grid_for(n_verts, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, stream>>>(coords, n_verts, rec);
    }
    return check_launch("fem_prepare_vertices");
}

extern "C" fem_status fem_integrate_laplacian_prepared(int dim, int64_t n_cells, int64_t n_verts,
                                                       const double *coords, const float *rec, const int32_t *conn,
                                                       const void *u, const void *K, int n_q, const double *qpts,
                                                       const double *qw, void *elem_out, fem_stream stream) {
    LapArgs a;
    fem_status st = fill_args(a, dim, n_cells, n_verts, coords, conn, u, K, n_q, qpts, qw, FEM_FP32_MIXED);
    if (st != FEM_OK) return st;
    if (n_cells == 0) return FEM_OK;
    if (!u || !K || !elem_out || !rec) return fail(FEM_ERR_ARG, "u, K, rec or elem_out is NULL");
    if ((reinterpret_cast<uintptr_t>(rec) & 31u) != 0) return fail(FEM_ERR_ARG, "rec must be 32-byte aligned");
    a.out = elem_out;
    const bool pairs = n_cells % 2 == 0 && aligned8(conn) && aligned8(K) && aligned8(elem_out);
    if (!pairs) return fail(FEM_ERR_SHAPE, "the prepared path needs an even cell count and 8-byte aligned rows");
    if (!(a.err = device_error_word())) return fail(FEM_ERR_CUDA, "device error word unavailable");
    const bool native_nq = (dim == 3 && n_q == 4) || (dim == 2 && n_q == 3);
    if (dim == 3) {
        auto k = native_nq ? lap_rec_kernel<3, 4> : lap_rec_kernel<3, 0>;
        launch_overlapped(k, resident_grid(reinterpret_cast<const void *>(k), kBlock, n_cells / 2), kBlock, 0, stream, a, rec);
    } else {
        auto k = native_nq ? lap_rec_kernel<2, 3> : lap_rec_kernel<2, 0>;
        launch_overlapped(k, resident_grid(reinterpret_cast<const void *>(k), kBlock, n_cells / 2), kBlock, 0, stream, a, rec);
    }
    return check_launch("fem_integrate_laplacian_prepared");
}
