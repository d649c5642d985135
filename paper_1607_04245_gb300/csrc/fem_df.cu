// fem_df.cu -- the Laplacian and linear-elasticity element residuals with float64 values
// and float64-class accuracy computed on the float32 pipe (FEM_FP64_DF).
//
// GB300 executes float32 FMAs ~68x faster than float64 ones (0.53 T float64 FMA/s
// against 35.9 T float32 FMA/s measured), so the float64 forms of these kernels are bound
// by the float64 pipe. This form keeps the inputs and outputs in float64 but carries every
// intermediate as an unevaluated pair of float32 values (hi + lo, a 47- to 48-bit
// significand; Dekker's double-length arithmetic built from TwoSum / TwoProduct):
//   * the Jacobian columns e_j = x_j - x_0 are formed in float64 (correctly rounded, no
//     loss to cancellation), then split into pairs with integer operations;
//   * u_b and K_q are split into pairs the same way and the weights are split on the host
//     (the Laplacian forms Kbar = sum_q w_q K_q in float64 and splits that instead);
//   * adjugate, determinant, field gradient, coefficient sum, the one division and the
//     contraction run in pair arithmetic, every sum of products as one compensated dot
//     product with a single renormalisation;
//   * each element-vector entry is widened back to float64 (integer operations) and
//     summed with one float64 add.
// Per cell (3D Laplacian) this issues 17 float64 operations instead of ~71 (the columns,
// the coefficient sum, the 4 outputs; elasticity: 21, the columns and 12 outputs). The
// relative error against the exact element integral stays near 1e-14 on the workloads
// (validated against the oracle at the float64 tolerance, 1e-12).
#include "fem_cell.cuh"

namespace fem {

struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl df_from_double(double x) {
    float hi, lo_u;
    split_f64(static_cast<uint32_t>(__double2loint(x)), static_cast<uint32_t>(__double2hiint(x)), hi, lo_u);
    return {hi, __fmul_rn(lo_u, 0x1p-23f)};
}

__device__ __forceinline__ dfl df_fast(float s, float e) {  // |s| >= |e|
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return df_fast(s, e);
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ dfl df_abs(dfl a) { return a.hi < 0.0f ? df_neg(a) : a; }

__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast(p, e);
}

// a / b: one float32 quotient, the remainder in pair arithmetic, a correction quotient
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const dfl r = df_sub(a, df_mul(b, dfl{q1, 0.0f}));
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return df_fast(q1, q2);
}

// Compensated sums of pair products, sum_i a_i b_i: the high parts of the products are
// added with TwoSum and every rounding error, with the cross terms a.hi b.lo + a.lo b.hi,
// goes into one float32 accumulator; one renormalisation at the end (Ogita, Rump and
// Oishi's Dot2 carried over to pair operands). The error stays at the pair precision,
// ~(n + 2) 2^-48 sum_i |a_i b_i|, for about 12 instead of 18 operations per term.
struct df_acc {
    float s, err;
};

__device__ __forceinline__ df_acc acc_first(dfl a, dfl b) {
    df_acc c;
    two_prod(a.hi, b.hi, c.s, c.err);
    c.err = fmaf(a.lo, b.hi, fmaf(a.hi, b.lo, c.err));
    return c;
}

__device__ __forceinline__ void acc_add(df_acc &c, dfl a, dfl b) {
    float p, ep, t;
    two_prod(a.hi, b.hi, p, ep);
    two_sum(c.s, p, c.s, t);
    c.err = fmaf(a.lo, b.hi, fmaf(a.hi, b.lo, __fadd_rn(c.err, __fadd_rn(t, ep))));
}

__device__ __forceinline__ dfl acc_value(df_acc c) {
    dfl r;
    two_sum(c.s, c.err, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ dfl df_dot2(dfl a0, dfl b0, dfl a1, dfl b1) {
    df_acc c = acc_first(a0, b0);
    acc_add(c, a1, b1);
    return acc_value(c);
}

__device__ __forceinline__ dfl df_dot3(dfl a0, dfl b0, dfl a1, dfl b1, dfl a2, dfl b2) {
    df_acc c = acc_first(a0, b0);
    acc_add(c, a1, b1);
    acc_add(c, a2, b2);
    return acc_value(c);
}

// adjugate rows n_j of the Jacobian with columns e_j, and det J = e_0 . n_0
template <int DIM>
__device__ __forceinline__ dfl df_adjugate(const dfl (&e)[DIM][DIM], dfl (&n)[DIM][DIM]) {
    if constexpr (DIM == 2) {
        n[0][0] = e[1][1], n[0][1] = df_neg(e[1][0]);
        n[1][0] = df_neg(e[0][1]), n[1][1] = e[0][0];
        return df_dot2(e[0][0], e[1][1], df_neg(e[0][1]), e[1][0]);
    } else {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const dfl *p = e[(j + 1) % 3], *q = e[(j + 2) % 3];
            n[j][0] = df_dot2(p[1], q[2], df_neg(p[2]), q[1]);
            n[j][1] = df_dot2(p[2], q[0], df_neg(p[0]), q[2]);
            n[j][2] = df_dot2(p[0], q[1], df_neg(p[1]), q[0]);
        }
        return df_dot3(e[0][0], n[0][0], e[0][1], n[0][1], e[0][2], n[0][2]);
    }
}

// n_j . h over DIM components
template <int DIM>
__device__ __forceinline__ dfl df_dotv(const dfl (&a)[DIM], const dfl (&b)[DIM]) {
    df_acc c = acc_first(a[0], b[0]);
#pragma unroll
    for (int i = 1; i < DIM; ++i) acc_add(c, a[i], b[i]);
    return acc_value(c);
}

// sum_j d_j n_j[i] for every component i
template <int DIM>
__device__ __forceinline__ void df_combine(const dfl (&d)[DIM], const dfl (&n)[DIM][DIM], dfl (&h)[DIM]) {
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        df_acc c = acc_first(d[0], n[0][i]);
#pragma unroll
        for (int j = 1; j < DIM; ++j) acc_add(c, d[j], n[j][i]);
        h[i] = acc_value(c);
    }
}

// sum_q w_q f_q for a float64 row f[q * C + c]
__device__ __forceinline__ dfl df_weighted(const float *whi, const float *wlo, const double *f, int64_t C, int64_t c,
                                           int nq) {
    df_acc acc = acc_first(dfl{whi[0], wlo[0]}, df_from_double(ld_stream(f + c)));
    for (int q = 1; q < nq; ++q) acc_add(acc, dfl{whi[q], wlo[q]}, df_from_double(ld_stream(f + q * C + c)));
    return acc_value(acc);
}

// sum_q w_q f_q for a float64 row f[q * C + c], in float64: one rounding per point, and a
// handful of float64-pipe instructions in place of the ~90 integer and float32 ones of the
// same sum in pair arithmetic
__device__ __forceinline__ double weighted64(const double *w, const double *f, int64_t C, int64_t c, int nq) {
    double s = w[0] * ld_stream(f + c);
    for (int q = 1; q < nq; ++q) s = fma(w[q], ld_stream(f + q * C + c), s);
    return s;
}

// float -> float64 with integer operations (normal numbers; zero and float32 subnormals,
// below 2^-126, widen to a signed zero)
__device__ __forceinline__ double widen(float x) {
    const uint32_t f = __float_as_uint(x);
    const uint32_t e8 = (f >> 23) & 0xffu;
    if (e8 == 0u) return __hiloint2double(static_cast<int>(f & 0x80000000u), 0);
    const uint32_t hi = (f & 0x80000000u) | ((e8 + 896u) << 20) | ((f & 0x7fffffu) >> 3);
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(f << 29));
}

__device__ __forceinline__ double df_to_double(dfl a) { return widen(a.hi) + widen(a.lo); }

struct DfArgs {
    const double *X[3];
    const int32_t *conn;
    const double *u, *K;
    double *out;
    int64_t C;
    uint32_t V;
    int nq;
    unsigned *err;  // device error word (FEM_DEVERR_BADMESH)
    double wd[FEM_MAX_QPTS];
};

template <int DIM>
__global__ void __launch_bounds__(kBlock, 5) lap_df_kernel(const __grid_constant__ DfArgs a) {
    pdl_wait();  // overlapped launch: the previous kernel's writes are visible from here
    pdl_trigger();
    constexpr int NB = DIM + 1;
    const int64_t C = a.C;
    const double *X[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) X[k] = a.X[k];
    uint32_t vmax = 0;     // largest vertex id seen (bad ids are clamped and reported)
    bool bad_det = false;  // a cell with det J = 0 or non-finite
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < C; c += stride) {
        uint32_t v[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) v[b] = clamp_vid(ld_stream(a.conn + b * C + c), a.V, vmax);
        // Kbar = sum_q w_q K_q in float64, then as a pair: 64 against 67 us on the
        // 1,572,864-tet workload. Forming u_j - u_0 in float64 too, or the elasticity and
        // adjoint coefficient sums in float64, was slower: the float64 pipe is half busy.
        const dfl kbar = df_from_double(weighted64(a.wd, a.K, C, c, a.nq));
        dfl du[DIM];
        {
            const dfl u0 = df_from_double(ld_gather(a.u + v[0]));
#pragma unroll
            for (int j = 0; j < DIM; ++j) du[j] = df_sub(df_from_double(ld_gather(a.u + v[j + 1])), u0);
        }
        // Jacobian columns in float64, then pairs
        double xs[NB][DIM];
        gather_coords<DIM>(X, v, xs);
        dfl e[DIM][DIM];
#pragma unroll
        for (int j = 0; j < DIM; ++j)
#pragma unroll
            for (int k = 0; k < DIM; ++k) e[j][k] = df_from_double(xs[j + 1][k] - xs[0][k]);
        // adjugate rows n_j and det J
        dfl n[DIM][DIM];
        const dfl det = df_adjugate<DIM>(e, n);
        bad_det |= det_bad(det.hi) | ids_repeat<NB>(v);
        // h = sum_j (u_j - u_0) n_j
        dfl h[DIM];
        df_combine<DIM>(du, n, h);
        // r_j = (Kbar / |det J|) n_j . h, r_0 = -(r_1 + ... + r_d)
        const dfl s = df_div(kbar, df_abs(det));
        dfl sum;
        double r[NB];
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
            const dfl rj = df_mul(s, df_dotv<DIM>(n[j], h));
            r[j + 1] = df_to_double(rj);
            sum = j == 0 ? rj : df_add(sum, rj);
        }
        r[0] = -df_to_double(sum);
#pragma unroll
        for (int b = 0; b < NB; ++b) __stcs(a.out + b * C + c, r[b]);
    }
    report_mesh(a.err, vmax, a.V, bad_det);
}

// called by fem_integrate_laplacian for FEM_FP64_DF (arguments already validated there)
fem_status launch_lap_df(int dim, int64_t n_cells, int64_t n_verts, const double *coords, const int32_t *conn,
                         const void *u, const void *K, int n_q, const double *qw, void *elem_out,
                         cudaStream_t stream) {
    DfArgs a;
    for (int k = 0; k < 3; ++k) a.X[k] = coords + (k < dim ? k : 0) * n_verts;
    a.conn = conn;
    a.u = static_cast<const double *>(u);
    a.K = static_cast<const double *>(K);
    a.out = static_cast<double *>(elem_out);
    a.C = n_cells;
    a.V = static_cast<uint32_t>(n_verts);
    a.nq = n_q;
    if (!(a.err = device_error_word())) return fail(FEM_ERR_CUDA, "device error word unavailable");
    for (int q = 0; q < FEM_MAX_QPTS; ++q) a.wd[q] = q < n_q ? qw[q] : 0.0;
    if (dim == 2) {
        auto k = lap_df_kernel<2>;
        launch_overlapped(k, grid_for(n_cells, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, stream, a);
    } else {
        auto k = lap_df_kernel<3>;
        launch_overlapped(k, grid_for(n_cells, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, stream, a);
    }
    return check_launch("fem_integrate_laplacian (FEM_FP64_DF)");
}

// ---- linear elasticity in the same form: f1 = lambda tr(eps) I + 2 mu eps. With the
// adjugate rows n_j and H[k][i] = sum_j (u_{j,k} - u_{0,k}) n_j[i] (grad u = H / det J):
//     T = Lbar tr(H) I + Mbar (H + H^T),  r_{b,k} = (T n_b)_k / |det J|,
// r_0 = -(r_1 + ... + r_d) per component; Lbar, Mbar the weighted sums of lambda and mu.

struct DfElArgs {
    const double *X[3];
    const int32_t *conn;
    const double *u, *lam, *mu;  // u [dim][V]; lam, mu [n_q][C]
    double *out;                 // [(dim+1)*dim][C]
    int64_t C;
    uint32_t V;
    int nq;
    unsigned *err;  // device error word (FEM_DEVERR_BADMESH)
    float whi[FEM_MAX_QPTS], wlo[FEM_MAX_QPTS];
};

// 3D: 4 CTAs per SM at up to 64 registers (73 unbounded, 3 CTAs: 190.3 -> 167.6 us on 2^21
// tets, steps back to back; 5 CTAs spill); 2D stays unbounded (59 registers, 4 CTAs).
template <int DIM>
constexpr int el_df_min_blocks() { return DIM == 3 ? 4 : 0; }  // 0: no minimum

template <int DIM>
__global__ void __launch_bounds__(kBlock, el_df_min_blocks<DIM>()) el_df_kernel(const __grid_constant__ DfElArgs a) {
    pdl_wait();  // overlapped launch: the previous kernel's writes are visible from here
    pdl_trigger();
    constexpr int NB = DIM + 1;
    const int64_t C = a.C;
    const int64_t V = a.V;
    const double *X[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) X[k] = a.X[k];
    uint32_t vmax = 0;     // largest vertex id seen (bad ids are clamped and reported)
    bool bad_det = false;  // a cell with det J = 0 or non-finite
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < C; c += stride) {
        uint32_t v[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) v[b] = clamp_vid(ld_stream(a.conn + b * C + c), a.V, vmax);
        // Lbar = sum_q w_q lambda_q, Mbar = sum_q w_q mu_q
        const dfl lbar = df_weighted(a.whi, a.wlo, a.lam, C, c, a.nq);
        const dfl mbar = df_weighted(a.whi, a.wlo, a.mu, C, c, a.nq);
        // Jacobian columns in float64, then pairs
        double xs[NB][DIM];
        gather_coords<DIM>(X, v, xs);
        dfl e[DIM][DIM];
#pragma unroll
        for (int j = 0; j < DIM; ++j)
#pragma unroll
            for (int k = 0; k < DIM; ++k) e[j][k] = df_from_double(xs[j + 1][k] - xs[0][k]);
        dfl n[DIM][DIM];
        const dfl det = df_adjugate<DIM>(e, n);
        bad_det |= det_bad(det.hi) | ids_repeat<NB>(v);
        // H[k][i] = sum_j (u_{j,k} - u_{0,k}) n_j[i]
        dfl H[DIM][DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const dfl u0 = df_from_double(ld_gather(a.u + k * V + v[0]));
            dfl du[DIM];
#pragma unroll
            for (int j = 0; j < DIM; ++j) du[j] = df_sub(df_from_double(ld_gather(a.u + k * V + v[j + 1])), u0);
            df_combine<DIM>(du, n, H[k]);
        }
        dfl tr = H[0][0];
#pragma unroll
        for (int k = 1; k < DIM; ++k) tr = df_add(tr, H[k][k]);
        const dfl inv = df_div(dfl{1.0f, 0.0f}, df_abs(det));
        // T is symmetric: its diagonal and upper entries, 1/|det J| folded into the Lame sums
        const dfl sm = df_mul(inv, mbar), sl = df_mul(df_mul(inv, lbar), tr);
        const dfl sm2{sm.hi + sm.hi, sm.lo + sm.lo};  // 2 sm, exact
        dfl Tm[DIM][DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            Tm[k][k] = df_add(df_mul(sm2, H[k][k]), sl);
#pragma unroll
            for (int i = k + 1; i < DIM; ++i) Tm[k][i] = Tm[i][k] = df_mul(sm, df_add(H[k][i], H[i][k]));
        }
        dfl r0[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) r0[k] = dfl{0.0f, 0.0f};
#pragma unroll
        for (int b = 1; b <= DIM; ++b)
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                const dfl rb = df_dotv<DIM>(Tm[k], n[b - 1]);
                r0[k] = df_sub(r0[k], rb);
                __stcs(a.out + (b * DIM + k) * C + c, df_to_double(rb));
            }
#pragma unroll
        for (int k = 0; k < DIM; ++k) __stcs(a.out + k * C + c, df_to_double(r0[k]));
    }
    report_mesh(a.err, vmax, a.V, bad_det);
}

// called by fem_integrate_elasticity for FEM_FP64_DF (arguments already validated there)
fem_status launch_el_df(int dim, int64_t n_cells, int64_t n_verts, const double *coords, const int32_t *conn,
                        const void *u, const void *lam, const void *mu, int n_q, const double *qw, void *elem_out,
                        cudaStream_t stream) {
    DfElArgs a;
    for (int k = 0; k < 3; ++k) a.X[k] = coords + (k < dim ? k : 0) * n_verts;
    a.conn = conn;
    a.u = static_cast<const double *>(u);
    a.lam = static_cast<const double *>(lam);
    a.mu = static_cast<const double *>(mu);
    a.out = static_cast<double *>(elem_out);
    a.C = n_cells;
    a.V = static_cast<uint32_t>(n_verts);
    a.nq = n_q;
    if (!(a.err = device_error_word())) return fail(FEM_ERR_CUDA, "device error word unavailable");
    for (int q = 0; q < FEM_MAX_QPTS; ++q) {
        const double w = q < n_q ? qw[q] : 0.0;
        a.whi[q] = static_cast<float>(w);
        a.wlo[q] = static_cast<float>(w - static_cast<double>(a.whi[q]));
    }
    if (dim == 2) {
        auto k = el_df_kernel<2>;
        launch_overlapped(k, grid_for(n_cells, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, stream, a);
    } else {
        auto k = el_df_kernel<3>;
        launch_overlapped(k, grid_for(n_cells, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, stream, a);
    }
    return check_launch("fem_integrate_elasticity (FEM_FP64_DF)");
}

// ---- the adjoint of the Laplacian residual in the same form: per element the residual of
// the adjoint weights lambda_e (scratch, summed per vertex afterwards) and
//     dK[q][e] = w_q (h_lambda . h_u) / |det J|.

struct DfAdjArgs {
    const double *X[3];
    const int32_t *conn;
    const double *u, *K, *lam;  // lam [dim+1][C]
    double *scratch, *dK;       // [dim+1][C], [n_q][C]
    int64_t C;
    uint32_t V;
    int nq;
    unsigned *err;  // device error word (FEM_DEVERR_BADMESH)
    float whi[FEM_MAX_QPTS], wlo[FEM_MAX_QPTS];
};

template <int DIM>
__global__ void __launch_bounds__(kBlock) adj_df_kernel(const __grid_constant__ DfAdjArgs a) {
    pdl_wait();  // overlapped launch: the previous kernel's writes are visible from here
    pdl_trigger();
    constexpr int NB = DIM + 1;
    const int64_t C = a.C;
    const double *X[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) X[k] = a.X[k];
    uint32_t vmax = 0;     // largest vertex id seen (bad ids are clamped and reported)
    bool bad_det = false;  // a cell with det J = 0 or non-finite
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < C; c += stride) {
        uint32_t v[NB];
        dfl uu[NB], ll[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            v[b] = clamp_vid(ld_stream(a.conn + b * C + c), a.V, vmax);
            uu[b] = df_from_double(ld_gather(a.u + v[b]));
            ll[b] = df_from_double(ld_stream(a.lam + b * C + c));
        }
        const dfl kbar = df_weighted(a.whi, a.wlo, a.K, C, c, a.nq);
        double xs[NB][DIM];
        gather_coords<DIM>(X, v, xs);
        dfl e[DIM][DIM];
#pragma unroll
        for (int j = 0; j < DIM; ++j)
#pragma unroll
            for (int k = 0; k < DIM; ++k) e[j][k] = df_from_double(xs[j + 1][k] - xs[0][k]);
        dfl n[DIM][DIM];
        const dfl det = df_adjugate<DIM>(e, n);
        bad_det |= det_bad(det.hi) | ids_repeat<NB>(v);
        // h_u = sum_j (u_j - u_0) n_j, h_l = sum_j (lambda_j - lambda_0) n_j
        dfl hu[DIM], hl[DIM], du[DIM], dl[DIM];
#pragma unroll
        for (int j = 0; j < DIM; ++j) du[j] = df_sub(uu[j + 1], uu[0]), dl[j] = df_sub(ll[j + 1], ll[0]);
        df_combine<DIM>(du, n, hu);
        df_combine<DIM>(dl, n, hl);
        const dfl inv = df_div(dfl{1.0f, 0.0f}, df_abs(det));
        const dfl s = df_mul(kbar, inv);
        // element residual of lambda_e: r_j = s n_j . h_l, r_0 = -(r_1 + ... + r_d)
        dfl sum;
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
            const dfl rj = df_mul(s, df_dotv<DIM>(n[j], hl));
            sum = j == 0 ? rj : df_add(sum, rj);
            __stcs(a.scratch + (j + 1) * C + c, df_to_double(rj));
        }
        __stcs(a.scratch + c, -df_to_double(sum));
        // dK[q] = w_q (h_l . h_u) / |det J|
        const dfl tf = df_mul(df_dotv<DIM>(hl, hu), inv);
        for (int q = 0; q < a.nq; ++q) __stcs(a.dK + q * C + c, df_to_double(df_mul(dfl{a.whi[q], a.wlo[q]}, tf)));
    }
    report_mesh(a.err, vmax, a.V, bad_det);
}

// the element part of fem_adjoint_laplacian for FEM_FP64_DF (arguments validated by the caller)
fem_status launch_adj_df(int dim, int64_t n_cells, int64_t n_verts, const double *coords, const int32_t *conn,
                         const void *u, const void *K, int n_q, const double *qw, const void *lambda, void *dK,
                         void *scratch, cudaStream_t stream) {
    DfAdjArgs a;
    for (int k = 0; k < 3; ++k) a.X[k] = coords + (k < dim ? k : 0) * n_verts;
    a.conn = conn;
    a.u = static_cast<const double *>(u);
    a.K = static_cast<const double *>(K);
    a.lam = static_cast<const double *>(lambda);
    a.scratch = static_cast<double *>(scratch);
    a.dK = static_cast<double *>(dK);
    a.C = n_cells;
    a.V = static_cast<uint32_t>(n_verts);
    a.nq = n_q;
    if (!(a.err = device_error_word())) return fail(FEM_ERR_CUDA, "device error word unavailable");
    for (int q = 0; q < FEM_MAX_QPTS; ++q) {
        const double w = q < n_q ? qw[q] : 0.0;
        a.whi[q] = static_cast<float>(w);
        a.wlo[q] = static_cast<float>(w - static_cast<double>(a.whi[q]));
    }
    if (dim == 2) {
        auto k = adj_df_kernel<2>;
        launch_overlapped(k, grid_for(n_cells, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, stream, a);
    } else {
        auto k = adj_df_kernel<3>;
        launch_overlapped(k, grid_for(n_cells, kBlock, reinterpret_cast<const void *>(k)), kBlock, 0, stream, a);
    }
    return check_launch("fem_adjoint_laplacian (FEM_FP64_DF)");
}

}  // namespace fem
