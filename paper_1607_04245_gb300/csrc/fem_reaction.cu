// fem_reaction.cu -- reaction-diffusion with an auxiliary coefficient field: the full
// bracket of Eq. 2 (both the f0 and the f1 term) with the pointwise functions of Eq. 8
// taking an auxiliary field a and its gradient:
//     f1(u, grad u, a) = a grad u,   f0(u, grad u, a, grad a) = c u + g grad a . grad u,
// a in P1 (nodal values, a(xi_q) = sum_b phi_b(xi_q) a_b) or in P0 (one value per cell,
// grad a = 0 inside the cell), c per quadrature point (optional), g a scalar (0: none).
//
// For P1 the gradients are constant on a cell, so the f1 part is the Laplacian element
// vector of fem_laplacian.cu with Kbar = sum_q w_q a(xi_q) = sum_b m_b a_b, where
// m_b = sum_q w_q phi_b(xi_q) (P1 a) or Kbar = a_e sum_q w_q (P0 a). The f0 part uses the
// basis tabulation phi_b(xi_q) (the matrix B of Eq. 2):
//     r_b += |det J| sum_q phi_b(xi_q) w_q c_q u(xi_q),  u(xi_q) = sum_a phi_a(xi_q) u_a,
// and, with grad u = h_u / det J and grad a = h_a / det J (h = sum_j (v_j - v_0) n_j over
// the adjugate rows n_j), the constant first-order term integrates to
//     r_b += m_b g (h_a . h_u) / |det J|.
#include <cmath>

#include "fem_cell.cuh"

namespace fem {

// P1 basis tabulation at the quadrature points and its weighted column sums
struct BasisTab {
    double phid[FEM_MAX_QPTS][4];
    float phif[FEM_MAX_QPTS][4];
    double md[4];
    float mf[4];
    double wsumd;
    float wsumf;
};

struct RdArgs {
    const double *X[3];
    const int32_t *conn;
    const void *u;
    const void *a;  // [V] (P1) or [C] (P0)
    const void *c;  // [n_q][C] or NULL
    void *out;      // [dim+1][C]
    int64_t C;
    uint32_t V;
    float tau2;
    double gd;  // g of the grad a term (P1 a only)
    float gf;
    unsigned *err;  // device error word (FEM_DEVERR_BADMESH)
    QuadW w;
    BasisTab t;
};

template <int P> __device__ __forceinline__ val_t<P> tab_phi(const BasisTab &t, int q, int b);
template <> __device__ __forceinline__ double tab_phi<FEM_FP64>(const BasisTab &t, int q, int b) { return t.phid[q][b]; }
template <> __device__ __forceinline__ float tab_phi<FEM_FP32_MIXED>(const BasisTab &t, int q, int b) { return t.phif[q][b]; }
template <> __device__ __forceinline__ float tab_phi<FEM_FP32>(const BasisTab &t, int q, int b) { return t.phif[q][b]; }

template <int P> __device__ __forceinline__ val_t<P> tab_m(const BasisTab &t, int b) {
    if constexpr (P == FEM_FP64) return t.md[b];
    else return t.mf[b];
}
template <int P> __device__ __forceinline__ val_t<P> tab_wsum(const BasisTab &t) {
    if constexpr (P == FEM_FP64) return t.wsumd;
    else return t.wsumf;
}
template <int P> __device__ __forceinline__ val_t<P> rd_weight(const QuadW &w, int q) {
    if constexpr (P == FEM_FP64) return w.wd[q];
    else return w.wf[q];
}

// f1 part (Laplacian with Kbar) and f0 part of one cell from its adjugate rows and det J;
// DRIFT: the grad a term, from the nodal values aa of a P1 coefficient
// num / |den|: quot_abs, or (NEWTON false, float64) the IEEE division
template <bool NEWTON, class T>
__device__ __forceinline__ T quot_div(T num, T den) {
    if constexpr (!NEWTON && std::is_same<T, double>::value) return num / fabs(den);
    else return quot_abs(num, den);
}

// NEWTON: the float64 quotients through quot_abs's Newton reciprocal (the float64 form);
// false in the mixed form's rare float64 recomputation, where the plain division keeps the
// main path's register allocation as it was
template <int DIM, int P, class T, bool REACT, bool DRIFT, int NQA, bool NEWTON = true>
__device__ __forceinline__ void rd_element(const RdArgs &a, const T (&n)[DIM][DIM], T det, const T (&uu)[DIM + 1],
                                           const T (&aa)[DIM + 1], T kbar, const T (&cq)[NQA], int nq,
                                           T (&r)[DIM + 1]) {
    constexpr int NB = DIM + 1;
    T h[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) h[i] = zero<T>();
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        const T du = uu[j + 1] - uu[0];
#pragma unroll
        for (int i = 0; i < DIM; ++i) h[i] = fma(du, n[j][i], h[i]);
    }
    // float64: one reciprocal of |det J| for both quotients (the float64 pipe bounds that
    // form); float32: two fast divisions (one reciprocal cost the mixed form 10 %)
    constexpr bool ONE_RCP = std::is_same<T, double>::value && NEWTON;
    const T y = ONE_RCP ? quot_abs(T(1), det) : T(0);
    const T s = ONE_RCP ? kbar * y : quot_div<NEWTON>(kbar, det);
    T sum = zero<T>();
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        r[j + 1] = s * dotv<DIM>(n[j], h);
        sum = sum + r[j + 1];
    }
    r[0] = -sum;
    if constexpr (DRIFT) {
        T ha[DIM];
#pragma unroll
        for (int i = 0; i < DIM; ++i) ha[i] = zero<T>();
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
            const T da = aa[j + 1] - aa[0];
#pragma unroll
            for (int i = 0; i < DIM; ++i) ha[i] = fma(da, n[j][i], ha[i]);
        }
        const T g = P == FEM_FP64 ? T(a.gd) : T(a.gf);
        const T t = ONE_RCP ? g * dotv<DIM>(ha, h) * y : quot_div<NEWTON>(g * dotv<DIM>(ha, h), det);
#pragma unroll
        for (int b = 0; b < NB; ++b) r[b] = fma(T(tab_m<P>(a.t, b)), t, r[b]);
    }
    if constexpr (REACT) {
        const T ad = det < T(0) ? -det : det;
        T m[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) m[b] = zero<T>();
        for (int q = 0; q < nq; ++q) {
            T uq = zero<T>();
#pragma unroll
            for (int b = 0; b < NB; ++b) uq = fma(T(tab_phi<P>(a.t, q, b)), uu[b], uq);
            const T tq = T(rd_weight<P>(a.w, q)) * cq[q] * uq;
#pragma unroll
            for (int b = 0; b < NB; ++b) m[b] = fma(T(tab_phi<P>(a.t, q, b)), tq, m[b]);
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) r[b] = fma(ad, m[b], r[b]);
    }
}

// Float64 recomputation of cell e of the mixed form (badly shaped, or a non-finite float32
// result), stored over the float32 element vector the caller has already written (same
// thread, program order). Everything is read again from global memory and summed in
// float64: the path is rare and kept out of line, so none of its state takes registers on
// the common path.
template <int DIM, bool A_P1, bool REACT, bool DRIFT>
__device__ __noinline__ void rd_fallback_store(const RdArgs &a, int64_t e) {
    constexpr int NB = DIM + 1;
    const int64_t C = a.C;
    const float *u = static_cast<const float *>(a.u);
    const float *af = static_cast<const float *>(a.a);
    const float *cf = static_cast<const float *>(a.c);
    uint32_t v[NB];
    double u64[NB], a64[NB], c64[FEM_MAX_QPTS];
    double kbar = 0.0;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        v[b] = clamp_vid(a.conn[b * C + e], a.V);
        u64[b] = u[v[b]];
        a64[b] = A_P1 ? double(af[v[b]]) : 0.0;
        if (A_P1) kbar += a.t.md[b] * a64[b];
    }
    if (!A_P1) kbar = a.t.wsumd * double(af[e]);
    if constexpr (REACT) {
        for (int q = 0; q < a.w.nq; ++q) c64[q] = cf[q * C + e];
    }
    const double *X[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) X[k] = a.X[k];
    double xs[NB][DIM], e64[DIM][DIM], n64[DIM][DIM], r64[NB];
    gather_coords<DIM>(X, v, xs);
    columns_f64<DIM>(xs, e64);
    const double det64 = adjugate_rows<DIM>(e64, n64);
    if (det_bad(det64) || ids_repeat<NB>(v)) record_device_error(a.err, FEM_DEVERR_BADMESH);
    rd_element<DIM, FEM_FP64, double, REACT, DRIFT, FEM_MAX_QPTS, false>(a, n64, det64, u64, a64, kbar, c64, a.w.nq,
                                                                        r64);
    float *out = static_cast<float *>(a.out);
#pragma unroll
    for (int b = 0; b < NB; ++b) out[b * C + e] = static_cast<float>(r64[b]);
}

// One cell: its vertex ids (unclamped), the P0 coefficient a0 (unused for a P1 field) and
// its reaction values ci at the quadrature points give the element vector rr. Returns
// false for a cell of the mixed form that fails its shape test (its rr is then
// meaningless; the caller recomputes it with rd_fallback_store). vmax and bad_det collect
// the mesh check (largest vertex id, det J = 0 or non-finite).
template <int DIM, int P, bool A_P1, bool REACT, bool DRIFT, int NQA>
__device__ __forceinline__ bool rd_cell(const RdArgs &a, const double *const (&X)[DIM], const int32_t (&vid)[DIM + 1],
                                        val_t<P> a0, const val_t<P> (&ci)[NQA], int nq, val_t<P> (&rr)[DIM + 1],
                                        uint32_t &vmax, bool &bad_det) {
    constexpr int NB = DIM + 1;
    using T = val_t<P>;
    const T *__restrict__ u = static_cast<const T *>(a.u);
    const T *__restrict__ af = static_cast<const T *>(a.a);
    uint32_t v[NB];
    T uu[NB], aa[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        v[b] = clamp_vid(vid[b], a.V, vmax);
        uu[b] = ld_gather(u + v[b]);
    }
    // Kbar = sum_q w_q a(xi_q)
    qsum_t<P> ks;
    if constexpr (A_P1) {
#pragma unroll
        for (int b = 0; b < NB; ++b) aa[b] = ld_gather(af + v[b]);
        ks.first(tab_m<P>(a.t, 0), aa[0]);
#pragma unroll
        for (int b = 1; b < NB; ++b) ks.add(tab_m<P>(a.t, b), aa[b]);
    } else {
#pragma unroll
        for (int b = 0; b < NB; ++b) aa[b] = zero<T>();
        ks.first(tab_wsum<P>(a.t), a0);
    }
    double xs[NB][DIM];
    gather_coords<DIM>(X, v, xs);
    if constexpr (P == FEM_FP64) {
        double ee[DIM][DIM], n[DIM][DIM];
        columns_f64<DIM>(xs, ee);
        const double det = adjugate_rows<DIM>(ee, n);
        bad_det |= det_bad(det) | ids_repeat<NB>(v);
        rd_element<DIM, P, double, REACT, DRIFT, NQA>(a, n, det, uu, aa, ks.value(), ci, nq, rr);
        return true;
    } else {
        float ee[DIM][DIM], n[DIM][DIM];
        if constexpr (P == FEM_FP32_MIXED) columns_mixed<DIM>(xs, ee);
        else columns_f32<DIM>(xs, ee);
        const float det = adjugate_rows<DIM>(ee, n);
        bool ok = true;
        if constexpr (P == FEM_FP32_MIXED) ok = shape_ok<DIM>(ee, det, a.tau2);
        else bad_det |= det_bad(det) | ids_repeat<NB>(v);
        rd_element<DIM, P, float, REACT, DRIFT, NQA>(a, n, det, uu, aa, ks.value(), ci, nq, rr);
        return ok;
    }
}

// Grid-stride over groups of CPT consecutive cells. A_P1: the coefficient field is nodal;
// DRIFT (P1 only): the grad a term. CPT = 4 with NQ > 0 (the quadrature size fixed at
// compile time) reads the connectivity, reaction and P0 coefficient rows and writes the
// element vectors with 16-byte vector accesses; CPT = 1, NQ = 0 is the general form
// (any n_q, unaligned rows, ragged sizes). Staging the rows through shared memory with the
// bulk-copy loop of the Laplacian kernel was slower here (37.2 against 33.7 us on the
// 1,572,864-tet workload): at that kernel's 2 CTAs per SM the register cap spills this
// element's state.
// 3D float32 forms take two cells per thread at 80 registers (3 CTAs of 256 threads per SM):
// 31.2 us on the 1,572,864-tet workload with reaction and drift, against 33.0 us with four
// cells at 128 registers (2 CTAs); 64 registers spill, and 2 CTAs of two cells run 39 us.
template <int DIM, int P, int CPT>
constexpr int rd_min_blocks() {
    return (P != FEM_FP64 && DIM == 3 && CPT == 2) ? 3 : 1;
}

template <int DIM, int P, bool A_P1, bool REACT, bool DRIFT, int CPT, int NQ>
__global__ void __launch_bounds__(kBlock, rd_min_blocks<DIM, P, CPT>()) rd_kernel(const __grid_constant__ RdArgs a) {
    pdl_wait();  // overlapped launch: the previous kernel's writes are visible from here
    pdl_trigger();
    static_assert(A_P1 || !DRIFT, "grad a vanishes inside a cell for a P0 field");
    static_assert(CPT == 1 || NQ > 0, "vector rows need a compile-time quadrature size");
    constexpr int NB = DIM + 1;
    constexpr int NQA = NQ > 0 ? NQ : FEM_MAX_QPTS;  // reaction values held per cell
    using T = val_t<P>;
    const int64_t C = a.C;
    const int nq = NQ > 0 ? NQ : a.w.nq;
    const T *__restrict__ af = static_cast<const T *>(a.a);
    const T *__restrict__ cf = static_cast<const T *>(a.c);
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
        T a0[CPT];
        if constexpr (!A_P1) load_row<CPT>(af + c0, a0);
        T cq[REACT ? NQA : 1][CPT];
        if constexpr (REACT) {
#pragma unroll(NQ > 0 ? NQ : 1)
            for (int q = 0; q < nq; ++q) load_row<CPT>(cf + q * C + c0, cq[q]);
        }
        T r[NB][CPT];
        bool ok[CPT];
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            int32_t vi[NB];
            T ci[NQA], rr[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) vi[b] = vid[b][i];
            if constexpr (REACT) {
#pragma unroll(NQ > 0 ? NQ : 1)
                for (int q = 0; q < nq; ++q) ci[q] = cq[q][i];
            }
            ok[i] = rd_cell<DIM, P, A_P1, REACT, DRIFT, NQA>(a, X, vi, A_P1 ? zero<T>() : a0[i], ci, nq, rr, vmax,
                                                            bad_det);
#pragma unroll
            for (int b = 0; b < NB; ++b) r[b][i] = rr[b];
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) store_row<CPT>(out + b * C + c0, r[b]);
        if constexpr (P == FEM_FP32_MIXED) {
#pragma unroll
            for (int i = 0; i < CPT; ++i)
                if (!ok[i]) rd_fallback_store<DIM, A_P1, REACT, DRIFT>(a, c0 + i);
        }
    }
    report_mesh(a.err, vmax, a.V, bad_det);
}

template <int DIM, int P, bool A_P1, bool REACT, bool DRIFT>
static void launch_rd_one(const RdArgs &a, bool vec4, bool vec2, cudaStream_t s) {
    constexpr int NQN = DIM + 1 == 4 ? 4 : 3;  // the workloads' rules: 3 points in 2D, 4 in 3D
    // float32 forms: two cells per thread in 3D, four in 2D (rd_min_blocks); the float64 form
    // is bound by the float64 pipe and keeps one cell per thread (four cost it occupancy: 457
    // against 416 us on the 1,572,864-tet workload)
    constexpr int CPTV = DIM == 3 ? 2 : 4;
    const bool vec = CPTV == 2 ? vec2 : vec4;
    if (P != FEM_FP64 && vec && a.w.nq == NQN) {
        auto k = rd_kernel<DIM, P, A_P1, REACT, DRIFT, CPTV, NQN>;
        launch_overlapped(k, grid_for((a.C + CPTV - 1) / CPTV, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, s, a);
    } else {
        auto k = rd_kernel<DIM, P, A_P1, REACT, DRIFT, 1, 0>;
        launch_overlapped(k, grid_for(a.C, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, s, a);
    }
}

template <int DIM, int P>
static fem_status launch_rd(const RdArgs &a, bool a_p1, bool react, bool drift, bool vec4, bool vec2,
                            cudaStream_t s) {
    if (a_p1) {
        if (drift) react ? launch_rd_one<DIM, P, true, true, true>(a, vec4, vec2, s)
                         : launch_rd_one<DIM, P, true, false, true>(a, vec4, vec2, s);
        else react ? launch_rd_one<DIM, P, true, true, false>(a, vec4, vec2, s)
                   : launch_rd_one<DIM, P, true, false, false>(a, vec4, vec2, s);
    } else {
        react ? launch_rd_one<DIM, P, false, true, false>(a, vec4, vec2, s) : launch_rd_one<DIM, P, false, false, false>(a, vec4, vec2, s);
    }
    return check_launch("fem_integrate_reaction_diffusion");
}

}  // namespace fem

using namespace fem;

extern "C" fem_status fem_integrate_reaction_diffusion(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                                       const int32_t *conn, const void *u, const void *a,
                                                       int a_space, const void *c, double drift, int n_q,
                                                       const double *qpts,
                                                       const double *qw, void *elem_out, fem_precision prec,
                                                       fem_stream stream) {
    fem_status st = check_common(dim, n_cells, n_verts, coords, conn);
    if (st != FEM_OK) return st;
    if (prec != FEM_FP64 && prec != FEM_FP32_MIXED && prec != FEM_FP32)
        return fail(FEM_ERR_ARG, "unknown precision %d", static_cast<int>(prec));
    if (a_space != 0 && a_space != 1) return fail(FEM_ERR_ARG, "a_space = %d, must be 0 (P0) or 1 (P1)", a_space);
    if (!std::isfinite(drift)) return fail(FEM_ERR_ARG, "drift must be finite");
    if (!qpts) return fail(FEM_ERR_ARG, "qpts is required: the f0 term and a P1 coefficient use phi_b(xi_q)");
    RdArgs r;
    if ((st = load_quadrature(dim, n_q, qpts, qw, r.w)) != FEM_OK) return st;
    if (n_cells == 0) return FEM_OK;
    if (!u || !a || !elem_out) return fail(FEM_ERR_ARG, "u, a or elem_out is NULL");
    // P1 basis at the quadrature points: phi_0 = 1 - sum_k xi_k, phi_b = xi_{b-1}
    for (int b = 0; b < 4; ++b) r.t.md[b] = 0.0;
    r.t.wsumd = 0.0;
    for (int q = 0; q < FEM_MAX_QPTS; ++q)
        for (int b = 0; b < 4; ++b) r.t.phid[q][b] = 0.0;
    for (int q = 0; q < n_q; ++q) {
        double s = 0.0;
        for (int k = 0; k < dim; ++k) s += qpts[q * dim + k];
        r.t.phid[q][0] = 1.0 - s;
        for (int b = 1; b <= dim; ++b) r.t.phid[q][b] = qpts[q * dim + b - 1];
        for (int b = 0; b <= dim; ++b) r.t.md[b] += qw[q] * r.t.phid[q][b];
        r.t.wsumd += qw[q];
    }
    for (int q = 0; q < FEM_MAX_QPTS; ++q)
        for (int b = 0; b < 4; ++b) r.t.phif[q][b] = static_cast<float>(r.t.phid[q][b]);
    for (int b = 0; b < 4; ++b) r.t.mf[b] = static_cast<float>(r.t.md[b]);
    r.t.wsumf = static_cast<float>(r.t.wsumd);
    for (int k = 0; k < 3; ++k) r.X[k] = coords + (k < dim ? k : 0) * n_verts;
    r.conn = conn;
    r.u = u;
    r.a = a;
    r.c = c;
    r.out = elem_out;
    r.C = n_cells;
    r.V = static_cast<uint32_t>(n_verts);
    const float tau = mixed_tau();
    r.tau2 = tau * tau;
    r.gd = drift;
    r.gf = static_cast<float>(drift);
    if (!(r.err = device_error_word())) return fail(FEM_ERR_CUDA, "device error word unavailable");
    // grad a vanishes inside a cell for a P0 field: the term is then absent
    const bool p1 = a_space == 1, react = c != nullptr, with_drift = p1 && drift != 0.0;
    // 16-byte rows: every cell-indexed array aligned and the cell count a multiple of 4
    const bool vec4 = n_cells % 4 == 0 && aligned16(conn) && aligned16(elem_out) && (!react || aligned16(c)) &&
                      (p1 || aligned16(a));
    const bool vec2 = n_cells % 2 == 0 && aligned8(conn) && aligned8(elem_out) && (!react || aligned8(c)) &&
                      (p1 || aligned8(a));
    switch (dim * 10 + static_cast<int>(prec)) {
        case 20: return launch_rd<2, FEM_FP64>(r, p1, react, with_drift, vec4, vec2, stream);
        case 21: return launch_rd<2, FEM_FP32_MIXED>(r, p1, react, with_drift, vec4, vec2, stream);
        case 22: return launch_rd<2, FEM_FP32>(r, p1, react, with_drift, vec4, vec2, stream);
        case 30: return launch_rd<3, FEM_FP64>(r, p1, react, with_drift, vec4, vec2, stream);
        case 31: return launch_rd<3, FEM_FP32_MIXED>(r, p1, react, with_drift, vec4, vec2, stream);
        case 32: return launch_rd<3, FEM_FP32>(r, p1, react, with_drift, vec4, vec2, stream);
    }
    return fail(FEM_ERR_ARG, "unsupported dim/precision");
}
