// fem_elasticity.cu -- element residual of P1 linear elasticity.
//
// Eq. 2 with f0 = 0 in its vector form (Sec. 2: f1 becomes a tensor) and the Lame
// stress f1 = lambda tr(eps) I + 2 mu eps, eps = (grad u + grad u^T)/2. For P1 the
// displacement gradient is constant on the cell: grad u = H / det J with
//     H[k][i] = sum_{j>=1} (u_{j,k} - u_{0,k}) n_j[i]
// (n_j the adjugate rows, fem_cell.cuh). The quadrature sum of the stress is
//     sum_q w_q sigma_q = T / det J,   T = Lbar tr(H) I + Mbar (H + H^T),
//     Lbar = sum_q w_q lambda_q,  Mbar = sum_q w_q mu_q,
// and the basis phase gives, for every basis function b and component k,
//     r_{b,k} = sum_q w_q |det J| sum_i sigma_q[k][i] G_b[i] = (T n_b)_k / |det J|,
// with r_0 = -(r_1 + ... + r_d) per component.
#include "fem_cell.cuh"

namespace fem {

struct ElArgs {
    const double *X[3];
    const int32_t *conn;
    const void *u;  // [dim][V]
    const void *lam;
    const void *mu;
    void *out;  // [(dim+1)*dim][C]
    int64_t C;
    uint32_t V;
    float tau2;
    unsigned *err;  // device error word (FEM_DEVERR_BADMESH)
    QuadW w;
};

template <int DIM, class T>
__device__ __forceinline__ void el_element(const T (&n)[DIM][DIM], T det, const T (&uu)[DIM + 1][DIM], T lbar,
                                           T mbar, T (&r)[DIM + 1][DIM]) {
    T H[DIM][DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k)
#pragma unroll
        for (int i = 0; i < DIM; ++i) H[k][i] = T(0);
#pragma unroll
    for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            T du = uu[j + 1][k] - uu[0][k];
#pragma unroll
            for (int i = 0; i < DIM; ++i) H[k][i] = fma(du, n[j][i], H[k][i]);
        }
    T tr = H[0][0];
#pragma unroll
    for (int k = 1; k < DIM; ++k) tr += H[k][k];
    T s;
    if constexpr (std::is_same<T, double>::value) s = quot_abs(1.0, det);
    else s = __fdividef(1.0f, fabsf(det));
    // T = s (Lbar tr(H) I + Mbar (H + H^T)) is symmetric: the diagonal and the d(d-1)/2
    // entries above it, with s folded into the two coefficients
    const T sm = s * mbar, sl = s * lbar * tr, sm2 = sm + sm;
    T Tm[DIM][DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        Tm[k][k] = fma(sm2, H[k][k], sl);
#pragma unroll
        for (int i = k + 1; i < DIM; ++i) Tm[k][i] = Tm[i][k] = sm * (H[k][i] + H[i][k]);
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) r[0][k] = T(0);
#pragma unroll
    for (int b = 1; b <= DIM; ++b)
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            r[b][k] = dotv<DIM>(Tm[k], n[b - 1]);
            r[0][k] -= r[b][k];
        }
}

template <int P>
__device__ __forceinline__ val_t<P> el_weight(const QuadW &w, int q) {
    if constexpr (P == FEM_FP64) return w.wd[q];
    else return w.wf[q];
}

// Float64 recomputation of cell c of the mixed form (badly shaped, or a non-finite float32
// result), stored over the float32 result the caller has already written (same thread,
// program order). Everything is read again from global memory and the coefficient sums
// come in as float64: the path is rare and kept out of line, so none of its state takes
// registers on the common path.
template <int DIM>
__device__ __noinline__ void el_fallback_store(const ElArgs &a, int64_t c, double lbar, double mbar) {
    constexpr int NB = DIM + 1;
    const int64_t C = a.C;
    const int64_t V = a.V;
    const float *u = static_cast<const float *>(a.u);
    uint32_t v[NB];
    double u64[NB][DIM];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        v[b] = clamp_vid(a.conn[b * C + c], a.V);
#pragma unroll
        for (int k = 0; k < DIM; ++k) u64[b][k] = u[k * V + v[b]];
    }
    const double *X[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) X[k] = a.X[k];
    double xs[NB][DIM], e64[DIM][DIM], n64[DIM][DIM], r64[NB][DIM];
    gather_coords<DIM>(X, v, xs);
    columns_f64<DIM>(xs, e64);
    const double det64 = adjugate_rows<DIM>(e64, n64);
    if (det_bad(det64) || ids_repeat<NB>(v)) record_device_error(a.err, FEM_DEVERR_BADMESH);
    el_element<DIM>(n64, det64, u64, lbar, mbar, r64);
    float *out = static_cast<float *>(a.out);
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int k = 0; k < DIM; ++k) out[(b * DIM + k) * C + c] = static_cast<float>(r64[b][k]);
}

// NQ > 0: quadrature size fixed at compile time, every coefficient row load issued
// before the first sum; NQ = 0: read from the arguments.
// Resident CTAs per SM the float32 forms are compiled for (their register cap): 2D with
// four cells per thread fits 64 registers (4 CTAs of 256 threads); 3D takes two cells per
// thread at 80 registers (3 CTAs). Measured on the workloads (2^22 triangles, 2^21 tets,
// L2 flushed): 2D 57.9 us at 80 registers (3 CTAs) -> 52.0 at 64; 3D 51.8 us with four cells
// per thread at 112 registers -> 46.0 with two at 80.
template <int DIM, int P, int CPT>
constexpr int el_min_blocks() {
    return P == FEM_FP64 ? 1 : (DIM == 2 && CPT == 4 ? 4 : (DIM == 3 && CPT == 2 ? 3 : 1));
}

template <int DIM, int P, int CPT, int NQ>
__global__ void __launch_bounds__(kBlock, el_min_blocks<DIM, P, CPT>()) el_kernel(const __grid_constant__ ElArgs a) {
    pdl_wait();  // overlapped launch: the previous kernel's writes are visible from here
    pdl_trigger();
    constexpr int NB = DIM + 1;
    using T = val_t<P>;
    const int64_t C = a.C;
    const T *__restrict__ u = static_cast<const T *>(a.u);
    const T *__restrict__ lam = static_cast<const T *>(a.lam);
    const T *__restrict__ mu = static_cast<const T *>(a.mu);
    T *__restrict__ out = static_cast<T *>(a.out);
    const double *X[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) X[k] = a.X[k];
    const int64_t V = a.V;

    uint32_t vmax = 0;     // largest vertex id seen (bad ids are clamped and reported)
    bool bad_det = false;  // a cell with det J = 0 or non-finite
    const int64_t ngroups = (C + CPT - 1) / CPT;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < ngroups; g += stride) {
        const int64_t c0 = g * CPT;
        int32_t vid[NB][CPT];
#pragma unroll
        for (int b = 0; b < NB; ++b) load_row<CPT>(a.conn + b * C + c0, vid[b]);

        qsum_t<P> ls[CPT], ms[CPT];
        if constexpr (NQ > 0) {
            T lq[NQ][CPT], mq[NQ][CPT];
#pragma unroll
            for (int q = 0; q < NQ; ++q) load_row<CPT>(lam + q * C + c0, lq[q]), load_row<CPT>(mu + q * C + c0, mq[q]);
#pragma unroll
            for (int i = 0; i < CPT; ++i)
                ls[i].first(el_weight<P>(a.w, 0), lq[0][i]), ms[i].first(el_weight<P>(a.w, 0), mq[0][i]);
#pragma unroll
            for (int q = 1; q < NQ; ++q)
#pragma unroll
                for (int i = 0; i < CPT; ++i)
                    ls[i].add(el_weight<P>(a.w, q), lq[q][i]), ms[i].add(el_weight<P>(a.w, q), mq[q][i]);
        } else {
            {
                T lq[CPT], mq[CPT];
                load_row<CPT>(lam + c0, lq);
                load_row<CPT>(mu + c0, mq);
                const T w0 = el_weight<P>(a.w, 0);
#pragma unroll
                for (int i = 0; i < CPT; ++i) ls[i].first(w0, lq[i]), ms[i].first(w0, mq[i]);
            }
            for (int q = 1; q < a.w.nq; ++q) {
                T lq[CPT], mq[CPT];
                load_row<CPT>(lam + q * C + c0, lq);
                load_row<CPT>(mu + q * C + c0, mq);
                const T wq = el_weight<P>(a.w, q);
#pragma unroll
                for (int i = 0; i < CPT; ++i) ls[i].add(wq, lq[i]), ms[i].add(wq, mq[i]);
            }
        }

        T r[NB * DIM][CPT];
        bool ok[CPT];
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            uint32_t v[NB];
            T uu[NB][DIM];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                v[b] = clamp_vid(vid[b][i], a.V, vmax);
#pragma unroll
                for (int k = 0; k < DIM; ++k) uu[b][k] = ld_gather(u + k * V + v[b]);
            }
            double xs[NB][DIM];
            gather_coords<DIM>(X, v, xs);
            T rr[NB][DIM];
            ok[i] = true;
            if constexpr (P == FEM_FP64) {
                double e[DIM][DIM], n[DIM][DIM];
                columns_f64<DIM>(xs, e);
                double det = adjugate_rows<DIM>(e, n);
                bad_det |= det_bad(det) | ids_repeat<NB>(v);
                el_element<DIM>(n, det, uu, ls[i].value(), ms[i].value(), rr);
            } else {
                float e[DIM][DIM], n[DIM][DIM];
                if constexpr (P == FEM_FP32_MIXED) columns_mixed<DIM>(xs, e);
                else columns_f32<DIM>(xs, e);
                float det = adjugate_rows<DIM>(e, n);
                if constexpr (P == FEM_FP32_MIXED) ok[i] = shape_ok<DIM>(e, det, a.tau2);
                else bad_det |= det_bad(det) | ids_repeat<NB>(v);
                // a failing cell's float32 result is meaningless here; it is recomputed below
                el_element<DIM>(n, det, uu, ls[i].value(), ms[i].value(), rr);
            }
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int k = 0; k < DIM; ++k) r[b * DIM + k][i] = rr[b][k];
        }
#pragma unroll
        for (int row = 0; row < NB * DIM; ++row) store_row<CPT>(out + row * C + c0, r[row]);
        if constexpr (P == FEM_FP32_MIXED) {
#pragma unroll
            for (int i = 0; i < CPT; ++i)
                if (!ok[i]) el_fallback_store<DIM>(a, c0 + i, ls[i].value_f64(), ms[i].value_f64());
        }
    }
    report_mesh(a.err, vmax, a.V, bad_det);
}

// vec4 / vec2: every cell-indexed row aligned for 16-byte / 8-byte accesses with four / two
// cells per thread
template <int DIM, int P>
static fem_status launch_el(const ElArgs &a, bool vec4, bool vec2, cudaStream_t s) {
    // 3D float32 forms: two cells per thread (four would hold 48 output registers until the
    // row stores); otherwise four
    constexpr int CPTV = (DIM == 3 && P != FEM_FP64) ? 2 : 4;
    const bool vec = CPTV == 2 ? vec2 : vec4;
    // the quadrature size of the workloads' rules (3 points in 2D, 4 in 3D) is compiled in.
    // The float32 forms run one wave of resident CTAs (steps back to back: 3D 52.9 -> 48.3
    // us, 2D 55.9 -> 54.6 us against up to 8 waves); float64 keeps the waves.
    if (vec && a.w.nq == DIM + 1) {
        auto k = el_kernel<DIM, P, CPTV, DIM + 1>;
        const int64_t n = (a.C + CPTV - 1) / CPTV;
        const void *kp = reinterpret_cast<const void *>(k);
        launch_overlapped(k, P == FEM_FP64 ? grid_for(n, kBlock, kp) : resident_grid(kp, kBlock, n), kBlock, 0, s, a);
    } else if (vec) {
        auto k = el_kernel<DIM, P, CPTV, 0>;
        launch_overlapped(k, grid_for((a.C + CPTV - 1) / CPTV, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, s, a);
    } else {
        auto k = el_kernel<DIM, P, 1, 0>;
        launch_overlapped(k, grid_for(a.C, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, s, a);
    }
    return check_launch("fem_integrate_elasticity");
}

}  // namespace fem

using namespace fem;

namespace fem {
fem_status launch_el_df(int dim, int64_t n_cells, int64_t n_verts, const double *coords, const int32_t *conn,
                        const void *u, const void *lam, const void *mu, int n_q, const double *qw, void *elem_out,
                        cudaStream_t stream);
}

extern "C" fem_status fem_integrate_elasticity(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                               const int32_t *conn, const void *u, const void *lam, const void *mu,
                                               int n_q, const double *qpts, const double *qw, void *elem_out,
                                               fem_precision prec, fem_stream stream) {
    fem_status st = check_common(dim, n_cells, n_verts, coords, conn);
    if (st != FEM_OK) return st;
    if (prec != FEM_FP64 && prec != FEM_FP32_MIXED && prec != FEM_FP32 && prec != FEM_FP64_DF)
        return fail(FEM_ERR_ARG, "unknown precision %d", static_cast<int>(prec));
    if (int64_t(dim) * n_verts >= (int64_t(1) << 31)) return fail(FEM_ERR_SHAPE, "too many vertices");
    ElArgs a;
    if ((st = load_quadrature(dim, n_q, qpts, qw, a.w)) != FEM_OK) return st;
    if (n_cells == 0) return FEM_OK;
    if (!u || !lam || !mu || !elem_out) return fail(FEM_ERR_ARG, "u, lam, mu or elem_out is NULL");
    if (prec == FEM_FP64_DF) return launch_el_df(dim, n_cells, n_verts, coords, conn, u, lam, mu, n_q, qw, elem_out,
                                                 stream);
    for (int k = 0; k < 3; ++k) a.X[k] = coords + (k < dim ? k : 0) * n_verts;
    a.conn = conn;
    a.u = u;
    a.lam = lam;
    a.mu = mu;
    a.out = elem_out;
    a.C = n_cells;
    a.V = static_cast<uint32_t>(n_verts);
    const float tau = mixed_tau();
    a.tau2 = tau * tau;
    if (!(a.err = device_error_word())) return fail(FEM_ERR_CUDA, "device error word unavailable");
    const bool vec4 = n_cells % 4 == 0 && aligned16(conn) && aligned16(lam) && aligned16(mu) && aligned16(elem_out);
    const bool vec2 = n_cells % 2 == 0 && aligned8(conn) && aligned8(lam) && aligned8(mu) && aligned8(elem_out);
    const int key = dim * 10 + static_cast<int>(prec);
    switch (key) {
        case 20: return launch_el<2, FEM_FP64>(a, vec4, vec2, stream);
        case 21: return launch_el<2, FEM_FP32_MIXED>(a, vec4, vec2, stream);
        case 22: return launch_el<2, FEM_FP32>(a, vec4, vec2, stream);
        case 30: return launch_el<3, FEM_FP64>(a, vec4, vec2, stream);
        case 31: return launch_el<3, FEM_FP32_MIXED>(a, vec4, vec2, stream);
        case 32: return launch_el<3, FEM_FP32>(a, vec4, vec2, stream);
    }
    return fail(FEM_ERR_ARG, "unsupported dim/precision");
}
