// fem_solver.cu -- matrix-free Jacobi-preconditioned conjugate-gradient solves with the
// assembled operators of Eq. 2: A v = E^T r_e(v), the element residuals of the
// variable-coefficient Laplacian or of linear elasticity summed into the vertices through
// the vertex-to-cell lists (fem_build_node2cell). Dirichlet vertices keep their value from
// the initial x. Also: mixed-precision iterative refinement around the FP32-mixed solve.
//
// Kernels here: the assembled diagonals (element stiffness diagonals summed per vertex), a
// deterministic two-level dot product, and the CG iteration in Chronopoulos and Gear's form
// with its scalars kept in device memory. The iteration loop runs on the device: one CG
// iteration is captured once into the body of a CUDA graph WHILE node, and the last kernel
// of the body counts the iteration and sets the loop condition (not converged and fewer
// than max_iter iterations). The host synchronises twice per solve (the initial residual
// norm, the final count) instead of once per iteration.
#include <cmath>
#include <cstring>
#include <mutex>

#include "fem_cell.cuh"

namespace fem {

fem_status launch_gather(int dim, int n_comp, int64_t C, int64_t V, const void *elem, const int32_t *node_ptr,
                         const int32_t *node_idx, void *out, fem_precision prec, cudaStream_t s);

constexpr int kDotBlocks = 1024;  // fixed: the partial sums and their order do not depend on the device

// element diagonals of the Laplacian stiffness: out[b][e] = Kbar |n_b|^2 / |det J|
template <int DIM, class T>
__global__ void lap_diag_kernel(const double *X0, int64_t C, uint32_t V, const int32_t *conn, const T *K, int nq,
                                QuadW w, T *out, unsigned *err) {
    constexpr int NB = DIM + 1;
    const double *X[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) X[k] = X0 + int64_t(k) * V;
    uint32_t vmax = 0;
    bool bad_det = false;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < C; e += stride) {
        uint32_t v[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) v[b] = clamp_vid(conn[b * C + e], V, vmax);
        double kbar = 0.0;
        for (int q = 0; q < nq; ++q) kbar += w.wd[q] * static_cast<double>(K[q * C + e]);
        double xs[NB][DIM], ee[DIM][DIM], n[DIM][DIM];
        gather_coords<DIM>(X, v, xs);
        columns_f64<DIM>(xs, ee);
        const double det = adjugate_rows<DIM>(ee, n);
        bad_det |= det_bad(det) | ids_repeat<NB>(v);
        const double s = kbar / fabs(det);
        double n0[DIM];
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            n0[i] = 0.0;
#pragma unroll
            for (int j = 0; j < DIM; ++j) n0[i] -= n[j][i];
        }
        out[e] = static_cast<T>(s * dotv<DIM>(n0, n0));
#pragma unroll
        for (int j = 0; j < DIM; ++j) out[(j + 1) * C + e] = static_cast<T>(s * dotv<DIM>(n[j], n[j]));
    }
    report_mesh(err, vmax, V, bad_det);
}

// element diagonals of the elasticity stiffness: for the unit displacement of component k at
// vertex b, H = e_k g^T with g = n_b (n_0 = -(n_1 + ... + n_d)), so
//     out[b*DIM + k][e] = (Lbar g_k^2 + Mbar (|g|^2 + g_k^2)) / |det J|
template <int DIM, class T>
__global__ void el_diag_kernel(const double *X0, int64_t C, uint32_t V, const int32_t *conn, const T *lam,
                               const T *mu, int nq, QuadW w, T *out, unsigned *err) {
    constexpr int NB = DIM + 1;
    const double *X[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) X[k] = X0 + int64_t(k) * V;
    uint32_t vmax = 0;
    bool bad_det = false;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < C; e += stride) {
        uint32_t v[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) v[b] = clamp_vid(conn[b * C + e], V, vmax);
        double lbar = 0.0, mbar = 0.0;
        for (int q = 0; q < nq; ++q) {
            lbar += w.wd[q] * static_cast<double>(lam[q * C + e]);
            mbar += w.wd[q] * static_cast<double>(mu[q * C + e]);
        }
        double xs[NB][DIM], ee[DIM][DIM], n[DIM][DIM];
        gather_coords<DIM>(X, v, xs);
        columns_f64<DIM>(xs, ee);
        const double det = adjugate_rows<DIM>(ee, n);
        bad_det |= det_bad(det) | ids_repeat<NB>(v);
        const double s = 1.0 / fabs(det);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            double g[DIM];
#pragma unroll
            for (int i = 0; i < DIM; ++i) {
                if (b == 0) {
                    g[i] = 0.0;
#pragma unroll
                    for (int j = 0; j < DIM; ++j) g[i] -= n[j][i];
                } else {
                    g[i] = n[b - 1][i];
                }
            }
            const double gg = dotv<DIM>(g, g);
#pragma unroll
            for (int k = 0; k < DIM; ++k)
                out[(b * DIM + k) * C + e] = static_cast<T>(s * (lbar * g[k] * g[k] + mbar * (gg + g[k] * g[k])));
        }
    }
    report_mesh(err, vmax, V, bad_det);
}

// block partial sums of x . y (float64 accumulation), fixed grid and order
template <class T>
__global__ void __launch_bounds__(256) dot_partial_kernel(int64_t n, const T *x, const T *y, double *partial) {
    __shared__ double s[256];
    double acc = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x; i < n; i += int64_t(kDotBlocks) * 256)
        acc += static_cast<double>(x[i]) * static_cast<double>(y[i]);
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

__global__ void __launch_bounds__(256) dot_final_kernel(const double *partial, double *result) {
    __shared__ double s[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < kDotBlocks; i += 256) acc += partial[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *result = s[0];
}

// scalars[] layout: 0 gamma = r.u, 1 delta = w.u, 2 alpha, 3 beta, 4 rr = r.r,
// 5 (rtol ||r_0||)^2, 6 iterations done, 7 the 32-bit block counter of the reduction
// (last_block), 8 alpha and beta rounded to float32 once (read by the float32 update)
enum { S_GAMMA = 0, S_DELTA = 1, S_ALPHA = 2, S_BETA = 3, S_RR = 4, S_TOL2 = 5, S_ITER = 6, S_TICKETS = 7,
       S_AB32 = 8, S_COUNT = 9 };

__device__ __forceinline__ unsigned *tickets(double *sc) { return reinterpret_cast<unsigned *>(sc + S_TICKETS); }

// Block-level sums of three doubles per thread (256 threads; sh: 3 x 256 doubles): a
// shared-memory tree, one barrier per level for the three; every thread gets the totals.
__device__ __forceinline__ void block_sum256x3(double (&v)[3], double *sh) {
#pragma unroll
    for (int m = 0; m < 3; ++m) sh[m * 256 + threadIdx.x] = v[m];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
#pragma unroll
            for (int m = 0; m < 3; ++m) sh[m * 256 + threadIdx.x] += sh[m * 256 + threadIdx.x + o];
        __syncthreads();
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) v[m] = sh[m * 256];
    __syncthreads();
}

// True in the block that finishes last: each block's thread 0 publishes the block's partial
// sums (fence), then takes a ticket; the block holding ticket kDotBlocks - 1 sees every
// partial and reduces them in place of a separate one-block kernel (the order of the sum
// does not depend on which block that is), then resets the counter for the next iteration.
__device__ __forceinline__ bool last_block(unsigned *ticket) {
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == unsigned(kDotBlocks - 1);
    }
    __syncthreads();
    return s_last;
}

// The loop is the conjugate gradient method in Chronopoulos and Gear's form (s-step CG with
// s = 1): with u = D^-1 r, w = A u and s = A p carried as vectors, both inner products of an
// iteration, gamma = r.u and delta = w.u, come from the same vectors at the same time, so an
// iteration is one vector update, one operator application and one reduction:
//     p = u + beta p,  s = w + beta s,  x += alpha p,  r -= alpha s,  u = r / D,
//     w = A u,  gamma' = r.u,  delta = w.u,
//     beta = gamma' / gamma,  alpha = gamma' / (delta - beta gamma' / alpha).
// The reductions visit the vertices with dot_partial_kernel's fixed grid and order (block b,
// thread t: i = 256 b + t + k 256 kDotBlocks) and are finished by the block that completes
// last, so every sum is reproducible and independent of the device.

// The vectors hold n_comp components per vertex, component-major ([n_comp][V]): entry i
// belongs to vertex i mod V, whose Dirichlet flag covers all its components.

// r = b - Ax on the free vertices (0 on fixed ones), u = D^-1 r, p = s = 0 (Dinv: the
// reciprocal of the Jacobi diagonal, formed once per solve by diag_fix_kernel)
template <class T>
__global__ void cg_init_kernel(int64_t N, int64_t V, const T *b, const T *Ax, const T *Dinv, const uint8_t *fixed,
                               T *r, T *u, T *p, T *sv) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += stride) {
        const T ri = fixed[i % V] ? T(0) : (b ? b[i] : T(0)) - Ax[i];
        r[i] = ri, u[i] = ri * Dinv[i], p[i] = T(0), sv[i] = T(0);
    }
}

// the product of two vector entries as a float64 term of a dot product: float32 entries are
// multiplied in float32 and widened once (one conversion on the float64 pipe instead of
// two and a float64 multiply); float64 entries multiply in float64
template <class T>
__device__ __forceinline__ double dot_term(T a, T b) {
    if constexpr (std::is_same<T, float>::value) return static_cast<double>(a * b);
    else return a * b;
}

// Inner products of float32 vectors without float64 arithmetic (the float64 pipe of this
// part issues 2 operations per clock per SM, against 128 float32): a double-float sum
// hi + lo, each product split exactly by TwoProduct and added by TwoSum (Knuth; the
// product of two float32 values is exact in the pair), the low parts summed in float32.
struct PairSum {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add_prod(float a, float b) {
        float p, e, s, t;
        two_prod(a, b, p, e);
        two_sum(hi, p, s, t);
        hi = s;
        lo += t + e;
    }
    __device__ __forceinline__ void merge(float h, float l) {
        float s, t;
        two_sum(hi, h, s, t);
        hi = s;
        lo += t + l;
    }
    __device__ __forceinline__ double value() const { return static_cast<double>(hi) + static_cast<double>(lo); }
};

// Warp tree of PairSums: lane 0 ends with the warp's total (fixed order: lane i takes lane
// i + o at o = 16, 8, 4, 2, 1).
__device__ __forceinline__ void warp_merge(PairSum &a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h = __shfl_down_sync(0xffffffffu, a.hi, o), l = __shfl_down_sync(0xffffffffu, a.lo, o);
        a.merge(h, l);
    }
}

// The totals of three PairSums per thread of a 256-thread block, in thread 0: warp trees,
// then the eight warp totals of each in a ninth (sh: 3 x 8 float2 of shared memory, free
// again on return; one barrier pair for the three).
__device__ __forceinline__ void block_merge256x3(PairSum (&a)[3], float2 *sh) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        warp_merge(a[m]);
        if (lane == 0) sh[m * 8 + (threadIdx.x >> 5)] = make_float2(a[m].hi, a[m].lo);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            PairSum b;
            if (lane < 8) b.hi = sh[m * 8 + lane].x, b.lo = sh[m * 8 + lane].y;
            warp_merge(b);
            a[m] = b;
        }
    }
    __syncthreads();
}

// p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = D^-1 r (in the vectors'
// own type). On fixed vertices r, u, w and so p and s stay 0, and x keeps its value.
template <class T>
__global__ void cg_update_kernel(int64_t N, const double *sc, const T *w, const T *Dinv, T *x, T *r, T *u, T *p,
                                 T *sv) {
    T alpha, beta;
    if constexpr (std::is_same<T, float>::value) {
        const float2 ab = *reinterpret_cast<const float2 *>(sc + S_AB32);  // no per-thread float64 conversion
        alpha = ab.x, beta = ab.y;
    } else {
        alpha = sc[S_ALPHA], beta = sc[S_BETA];
    }
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += stride) {
        const T pi = u[i] + beta * p[i];
        const T si = w[i] + beta * sv[i];
        p[i] = pi;
        sv[i] = si;
        x[i] = x[i] + alpha * pi;
        const T ri = r[i] - alpha * si;
        r[i] = ri;
        u[i] = ri * Dinv[i];
    }
}

// w = A u: the element vectors of u summed per vertex in list order (as the nodal gather
// does), 0 on fixed vertices; with the block partial sums of r.u, w.u and r.r. The block
// that finishes last forms gamma, delta and rr and the next alpha and beta; INIT (before
// the loop): alpha = gamma / delta, beta = 0; otherwise it also counts the iteration and
// sets the loop condition (not converged, fewer than max_iter; a NaN residual ends the loop:
// every comparison with it is false).
template <int NB, int NCOMP, class T, bool INIT>
__global__ void __launch_bounds__(256) cg_apply_dots_kernel(int64_t C, int64_t V, const T *__restrict__ elem,
                                                            const int32_t *__restrict__ ptr,
                                                            const int32_t *__restrict__ idx, const uint8_t *fixed,
                                                            const T *r, const T *u, T *w, double *partial, double *sc,
                                                            int max_iter, cudaGraphConditionalHandle loop) {
    constexpr bool F32 = std::is_same<T, float>::value;
    __shared__ double sh[F32 ? 1 : 3 * 256];
    __shared__ float2 sh2[3 * 8];
    // list entry t = NB cell + a: element row (a, component k)
    auto entry = [&](int32_t t, int k) {
        const int32_t cell = t / NB, a = t - cell * NB;
        return __ldg(elem + int64_t(a * NCOMP + k) * C + cell);
    };
    double ru = 0.0, wu = 0.0, rr = 0.0;  // float64 vectors
    PairSum pd[3];                         // float32 vectors: r.u, w.u, r.r
    for (int64_t n = int64_t(blockIdx.x) * 256 + threadIdx.x; n < V; n += int64_t(kDotBlocks) * 256) {
        const int32_t b = ptr[n], e = ptr[n + 1];
        NodeSum<T> acc[NCOMP];
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
        const bool fx = fixed[n] != 0;
#pragma unroll
        for (int k = 0; k < NCOMP; ++k) {
            const int64_t i = int64_t(k) * V + n;
            const T wn = fx ? T(0) : acc[k].value();
            w[i] = wn;
            const T rn = r[i], un = u[i];
            if constexpr (F32) {
                pd[0].add_prod(rn, un);
                pd[1].add_prod(wn, un);
                pd[2].add_prod(rn, rn);
            } else {
                ru += dot_term(rn, un);
                wu += dot_term(wn, un);
                rr += dot_term(rn, rn);
            }
        }
    }
    double gamma = 0.0, delta = 0.0, rrs = 0.0;  // the totals, in thread 0 of the last block
    if constexpr (F32) {
        // block partials as (hi, lo) pairs in place of the float64 partials
        float2 *pp = reinterpret_cast<float2 *>(partial);
        block_merge256x3(pd, sh2);
        if (threadIdx.x == 0)
            for (int m = 0; m < 3; ++m) pp[m * kDotBlocks + blockIdx.x] = make_float2(pd[m].hi, pd[m].lo);
        if (!last_block(tickets(sc))) return;
        PairSum at[3];
        for (int i = threadIdx.x; i < kDotBlocks; i += 256)
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const float2 v = __ldcg(pp + m * kDotBlocks + i);
                at[m].merge(v.x, v.y);
            }
        block_merge256x3(at, sh2);
        gamma = at[0].value(), delta = at[1].value(), rrs = at[2].value();
    } else {
        double t[3] = {ru, wu, rr};
        block_sum256x3(t, sh);
        if (threadIdx.x == 0)
            for (int m = 0; m < 3; ++m) partial[m * kDotBlocks + blockIdx.x] = t[m];
        if (!last_block(tickets(sc))) return;
        double at[3] = {0.0, 0.0, 0.0};
        for (int i = threadIdx.x; i < kDotBlocks; i += 256)
#pragma unroll
            for (int m = 0; m < 3; ++m) at[m] += __ldcg(partial + m * kDotBlocks + i);
        block_sum256x3(at, sh);
        gamma = at[0], delta = at[1], rrs = at[2];
    }
    if (threadIdx.x == 0) {
        if constexpr (INIT) {
            sc[S_ALPHA] = delta != 0.0 ? gamma / delta : 0.0;
            sc[S_BETA] = 0.0;
        } else {
            const double g0 = sc[S_GAMMA], a_old = sc[S_ALPHA];
            const double beta = g0 != 0.0 ? gamma / g0 : 0.0;
            const double den = a_old != 0.0 ? delta - beta * gamma / a_old : delta;
            sc[S_BETA] = beta;
            sc[S_ALPHA] = den != 0.0 ? gamma / den : 0.0;
            const double it = sc[S_ITER] + 1.0;
            sc[S_ITER] = it;
            const bool more = it < static_cast<double>(max_iter) && rrs > sc[S_TOL2] && rrs > 0.0;
            cudaGraphSetConditional(loop, more ? 1u : 0u);
        }
        *reinterpret_cast<float2 *>(sc + S_AB32) =
            make_float2(static_cast<float>(sc[S_ALPHA]), static_cast<float>(sc[S_BETA]));
        sc[S_GAMMA] = gamma;
        sc[S_DELTA] = delta;
        sc[S_RR] = rrs;
        tickets(sc)[0] = 0u;
    }
}

__global__ void loop_init_kernel(double *sc, double tol2) {
    sc[S_TOL2] = tol2;
    sc[S_ITER] = 0.0;
}

// a library stream per device to capture the loop body on (capture needs a stream other
// than the legacy default one, which callers may pass)
static cudaStream_t capture_stream() {
    static std::mutex mu;
    static cudaStream_t per_dev[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!per_dev[dev] && cudaStreamCreateWithFlags(&per_dev[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        per_dev[dev] = nullptr;
    }
    return per_dev[dev];
}

// fixed vertices get D = 1 (their rows are the identity); then D is replaced by its
// reciprocal, so that every application of the preconditioner is one multiply
template <class T>
__global__ void diag_fix_kernel(int64_t N, int64_t V, const uint8_t *fixed, T *D) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += stride)
        D[i] = (fixed[i % V] || !(D[i] > T(0))) ? T(1) : T(1) / D[i];
}

static size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

struct Workspace {
    void *elem, *D, *r, *z, *p, *q, *sv;  // D holds D^-1, z holds u = D^-1 r, q holds w = A u, sv s = A p
    double *partial, *scalars;
};

static size_t carve(int64_t C, int64_t V, int dim, size_t vs, void *base, Workspace *w, int ncomp = 1) {
    size_t off = 0;
    char *b = static_cast<char *>(base);
    auto take = [&](size_t bytes) {
        void *p = b ? b + off : nullptr;
        off += align256(bytes);
        return p;
    };
    const size_t N = size_t(ncomp) * size_t(V);
    void *elem = take(size_t(dim + 1) * size_t(ncomp) * size_t(C) * vs);
    void *D = take(N * vs), *r = take(N * vs), *z = take(N * vs);
    void *p = take(N * vs), *q = take(N * vs), *sv = take(N * vs);
    double *partial = static_cast<double *>(take(sizeof(double) * 3 * kDotBlocks));
    double *scalars = static_cast<double *>(take(sizeof(double) * S_COUNT));
    if (w) *w = Workspace{elem, D, r, z, p, q, sv, partial, scalars};
    return off;
}

// the assembled operator of a solve: the Laplacian with K, or elasticity with lambda, mu
struct Operator {
    int physics;  // 0 Laplacian, 1 elasticity
    const void *K, *lam, *mu;
    int ncomp(int dim) const { return physics == 0 ? 1 : dim; }
};

template <class T>
static fem_status pcg_run(int dim, int64_t C, int64_t V, const double *coords, const int32_t *conn,
                          const Operator &op, int n_q, const double *qpts, const double *qw, const int32_t *ptr,
                          const int32_t *idx, const uint8_t *fixed, const void *b, void *x, int max_iter,
                          double rtol, const Workspace &w, int *iters_out, double *resid_out, fem_precision prec,
                          cudaStream_t s, bool diag_ready = false) {
    // the residual runs in `prec`; every other kernel sees the value type (FEM_FP64_DF
    // values are float64). diag_ready: w.D already holds the reciprocal of this operator's
    // diagonal (a repeated solve with the same workspace).
    const fem_precision vprec = prec == FEM_FP64_DF ? FEM_FP64 : prec;
    T *X = static_cast<T *>(x);
    T *D = static_cast<T *>(w.D), *r = static_cast<T *>(w.r), *z = static_cast<T *>(w.z);
    T *p = static_cast<T *>(w.p), *q = static_cast<T *>(w.q), *sv = static_cast<T *>(w.sv);
    const T *B = static_cast<const T *>(b);
    const int nc = op.ncomp(dim);
    const int64_t N = int64_t(nc) * V;  // unknowns
    const int gV = static_cast<int>(std::min<int64_t>((N + 255) / 256, 4096));
    QuadW qwt;
    fem_status st = load_quadrature(dim, n_q, qpts, qw, qwt);
    if (st != FEM_OK) return st;
    // assembled diagonal
    if (!diag_ready) {
        const int g = static_cast<int>(std::min<int64_t>((C + 255) / 256, 4096));
        unsigned *err = device_error_word();
        if (!err) return fail(FEM_ERR_CUDA, "device error word unavailable");
        const uint32_t V32 = static_cast<uint32_t>(V);
        T *el = static_cast<T *>(w.elem);
        if (op.physics == 0) {
            const T *K = static_cast<const T *>(op.K);
            if (dim == 2) lap_diag_kernel<2, T><<<g, 256, 0, s>>>(coords, C, V32, conn, K, n_q, qwt, el, err);
            else lap_diag_kernel<3, T><<<g, 256, 0, s>>>(coords, C, V32, conn, K, n_q, qwt, el, err);
        } else {
            const T *lam = static_cast<const T *>(op.lam), *mu = static_cast<const T *>(op.mu);
            if (dim == 2) el_diag_kernel<2, T><<<g, 256, 0, s>>>(coords, C, V32, conn, lam, mu, n_q, qwt, el, err);
            else el_diag_kernel<3, T><<<g, 256, 0, s>>>(coords, C, V32, conn, lam, mu, n_q, qwt, el, err);
        }
        if ((st = check_launch("fem_pcg diagonal")) != FEM_OK) return st;
        if ((st = launch_gather(dim, nc, C, V, w.elem, ptr, idx, D, vprec, s)) != FEM_OK) return st;
        diag_fix_kernel<T><<<gV, 256, 0, s>>>(N, V, fixed, D);
    }
    // the element vectors of v in w.elem
    auto residual = [&](const T *v, cudaStream_t cs) -> fem_status {
        if (op.physics == 0)
            return fem_integrate_laplacian(dim, C, V, coords, conn, v, op.K, n_q, qpts, qw, w.elem, prec, cs);
        return fem_integrate_elasticity(dim, C, V, coords, conn, v, op.lam, op.mu, n_q, qpts, qw, w.elem, prec, cs);
    };
    auto matvec = [&](const T *v, T *out, cudaStream_t cs) -> fem_status {
        fem_status e = residual(v, cs);
        if (e != FEM_OK) return e;
        return launch_gather(dim, nc, C, V, w.elem, ptr, idx, out, vprec, cs);
    };
    // w = A u (0 on fixed vertices) with the iteration's inner products and scalars
    auto apply_dots = [&](bool init, cudaGraphConditionalHandle loop, cudaStream_t cs) -> fem_status {
        fem_status e = residual(z, cs);
        if (e != FEM_OK) return e;
        const T *el = static_cast<const T *>(w.elem);
        const int mi = init ? 0 : max_iter;
        auto go = [&](auto kern) {
            kern<<<kDotBlocks, 256, 0, cs>>>(C, V, el, ptr, idx, fixed, r, z, q, w.partial, w.scalars, mi, loop);
        };
        const int key = dim * 10 + nc;  // 21 22 31 33
        if (init) {
            if (key == 21) go(cg_apply_dots_kernel<3, 1, T, true>);
            else if (key == 22) go(cg_apply_dots_kernel<3, 2, T, true>);
            else if (key == 31) go(cg_apply_dots_kernel<4, 1, T, true>);
            else go(cg_apply_dots_kernel<4, 3, T, true>);
        } else {
            if (key == 21) go(cg_apply_dots_kernel<3, 1, T, false>);
            else if (key == 22) go(cg_apply_dots_kernel<3, 2, T, false>);
            else if (key == 31) go(cg_apply_dots_kernel<4, 1, T, false>);
            else go(cg_apply_dots_kernel<4, 3, T, false>);
        }
        return FEM_OK;
    };
    auto read = [&](int slot, int n, double *v) -> fem_status {
        cudaError_t e = cudaMemcpyAsync(v, w.scalars + slot, n * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(FEM_ERR_CUDA, "fem_pcg_laplacian: %s", cudaGetErrorString(e));
        return FEM_OK;
    };
    // r0 = b - A x0 on the free vertices, u0 = D^-1 r0, w0 = A u0, gamma0, delta0, alpha0
    {
        const cudaError_t e = cudaMemsetAsync(w.scalars, 0, sizeof(double) * S_COUNT, s);
        if (e != cudaSuccess) return fail(FEM_ERR_CUDA, "fem_pcg_laplacian: %s", cudaGetErrorString(e));
    }
    if ((st = matvec(X, q, s)) != FEM_OK) return st;
    cg_init_kernel<T><<<gV, 256, 0, s>>>(N, V, B, q, D, fixed, r, z, p, sv);
    if ((st = apply_dots(true, 0, s)) != FEM_OK) return st;
    double rr0 = 0.0;
    if ((st = read(S_RR, 1, &rr0)) != FEM_OK) return st;
    const double r0 = std::sqrt(rr0);
    double rn = r0;
    int it = 0;
    if (max_iter > 0 && rn > rtol * r0 && rn > 0.0) {
        const double tol = rtol * r0;
        loop_init_kernel<<<1, 1, 0, s>>>(w.scalars, tol * tol);
        // the loop: a graph holding one WHILE node whose body is one CG iteration
        cudaStream_t cs = capture_stream();
        if (!cs) return fail(FEM_ERR_CUDA, "fem_pcg_laplacian: no capture stream");
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaGraphConditionalHandle loop = 0;
        cudaError_t e = cudaGraphCreate(&graph, 0);
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&loop, graph, 1u, cudaGraphCondAssignDefault);
        cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
        np.conditional.handle = loop;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
        // one capture at a time on the shared capture stream
        static std::mutex capture_mu;
        std::unique_lock<std::mutex> capture_lock(capture_mu);
        if (e == cudaSuccess)
            e = cudaStreamBeginCaptureToGraph(cs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            // one iteration in 3 kernels: the vector updates; the residual of u; w = A u with
            // the inner products, the scalars and the loop condition
            cg_update_kernel<T><<<gV, 256, 0, cs>>>(N, w.scalars, q, D, X, r, z, p, sv);
            st = apply_dots(false, loop, cs);
            cudaGraph_t body = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(cs, &body);
            if (e2 != cudaSuccess) e = e2;
        }
        capture_lock.unlock();
        if (e == cudaSuccess && st == FEM_OK) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e == cudaSuccess && st == FEM_OK) e = cudaGraphLaunch(exec, s);
        if (e == cudaSuccess && st == FEM_OK) e = cudaStreamSynchronize(s);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (st != FEM_OK) return st;
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(FEM_ERR_CUDA, "fem_pcg_laplacian (iteration graph): %s", cudaGetErrorString(e));
        }
        double tail[3];  // rr, tol^2, iterations
        if ((st = read(S_RR, 3, tail)) != FEM_OK) return st;
        rn = std::sqrt(tail[0]);
        it = static_cast<int>(tail[2]);
    }
    if ((st = check_launch("fem_pcg_laplacian")) != FEM_OK) return st;
    if (iters_out) *iters_out = it;
    if (resid_out) *resid_out = r0 > 0.0 ? rn / r0 : 0.0;
    return FEM_OK;
}

}  // namespace fem

using namespace fem;

extern "C" int64_t fem_pcg_work_bytes(int dim, int64_t n_cells, int64_t n_verts, fem_precision prec) {
    if ((dim != 2 && dim != 3) || n_cells < 0 || n_verts < 0) return -1;
    const size_t vs = prec == FEM_FP64 || prec == FEM_FP64_DF ? 8 : 4;
    return static_cast<int64_t>(carve(n_cells, n_verts, dim, vs, nullptr, nullptr));
}

extern "C" fem_status fem_pcg_laplacian(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                        const int32_t *conn, const void *K, int n_q, const double *qpts,
                                        const double *qw, const int32_t *node_ptr, const int32_t *node_idx,
                                        const uint8_t *fixed, const void *b, void *x, int max_iter, double rtol,
                                        void *work, int64_t work_bytes, int *iters_out, double *resid_out,
                                        fem_precision prec, fem_stream stream) {
    fem_status st = check_common(dim, n_cells, n_verts, coords, conn);
    if (st != FEM_OK) return st;
    if (prec != FEM_FP64 && prec != FEM_FP32_MIXED && prec != FEM_FP32 && prec != FEM_FP64_DF)
        return fail(FEM_ERR_ARG, "unknown precision %d", static_cast<int>(prec));
    if (max_iter < 0 || !(rtol >= 0.0)) return fail(FEM_ERR_ARG, "max_iter must be >= 0 and rtol >= 0");
    if (n_verts == 0) {
        if (iters_out) *iters_out = 0;
        if (resid_out) *resid_out = 0.0;
        return FEM_OK;
    }
    if (!K || !node_ptr || !node_idx || !fixed || !x || !work) return fail(FEM_ERR_ARG, "a NULL array argument");
    const int64_t need = fem_pcg_work_bytes(dim, n_cells, n_verts, prec);
    if (work_bytes < need)
        return fail(FEM_ERR_OOM, "fem_pcg_laplacian: workspace of %lld bytes, %lld needed",
                    static_cast<long long>(work_bytes), static_cast<long long>(need));
    if (reinterpret_cast<uintptr_t>(work) & 255u) return fail(FEM_ERR_ARG, "work must be 256-byte aligned");
    Workspace w;
    const bool f64 = prec == FEM_FP64 || prec == FEM_FP64_DF;
    carve(n_cells, n_verts, dim, f64 ? 8 : 4, work, &w);
    if (f64)
        return pcg_run<double>(dim, n_cells, n_verts, coords, conn, Operator{0, K, nullptr, nullptr}, n_q, qpts, qw,
                               node_ptr, node_idx, fixed, b, x,
                               max_iter, rtol, w, iters_out, resid_out, prec, stream);
    return pcg_run<float>(dim, n_cells, n_verts, coords, conn, Operator{0, K, nullptr, nullptr}, n_q, qpts, qw,
                          node_ptr, node_idx, fixed, b, x,
                          max_iter, rtol, w, iters_out, resid_out, prec, stream);
}

extern "C" int64_t fem_pcg_elasticity_work_bytes(int dim, int64_t n_cells, int64_t n_verts, fem_precision prec) {
    if ((dim != 2 && dim != 3) || n_cells < 0 || n_verts < 0) return -1;
    const size_t vs = prec == FEM_FP64 || prec == FEM_FP64_DF ? 8 : 4;
    return static_cast<int64_t>(carve(n_cells, n_verts, dim, vs, nullptr, nullptr, dim));
}

extern "C" fem_status fem_pcg_elasticity(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                         const int32_t *conn, const void *lam, const void *mu, int n_q,
                                         const double *qpts, const double *qw, const int32_t *node_ptr,
                                         const int32_t *node_idx, const uint8_t *fixed, const void *b, void *x,
                                         int max_iter, double rtol, void *work, int64_t work_bytes, int *iters_out,
                                         double *resid_out, fem_precision prec, fem_stream stream) {
    fem_status st = check_common(dim, n_cells, n_verts, coords, conn);
    if (st != FEM_OK) return st;
    if (prec != FEM_FP64 && prec != FEM_FP32_MIXED && prec != FEM_FP32 && prec != FEM_FP64_DF)
        return fail(FEM_ERR_ARG, "unknown precision %d", static_cast<int>(prec));
    if (max_iter < 0 || !(rtol >= 0.0)) return fail(FEM_ERR_ARG, "max_iter must be >= 0 and rtol >= 0");
    if (int64_t(dim) * n_verts >= (int64_t(1) << 31)) return fail(FEM_ERR_SHAPE, "too many vertices");
    if (n_verts == 0) {
        if (iters_out) *iters_out = 0;
        if (resid_out) *resid_out = 0.0;
        return FEM_OK;
    }
    if (!lam || !mu || !node_ptr || !node_idx || !fixed || !x || !work)
        return fail(FEM_ERR_ARG, "a NULL array argument");
    const int64_t need = fem_pcg_elasticity_work_bytes(dim, n_cells, n_verts, prec);
    if (work_bytes < need)
        return fail(FEM_ERR_OOM, "fem_pcg_elasticity: workspace of %lld bytes, %lld needed",
                    static_cast<long long>(work_bytes), static_cast<long long>(need));
    if (reinterpret_cast<uintptr_t>(work) & 255u) return fail(FEM_ERR_ARG, "work must be 256-byte aligned");
    Workspace w;
    const bool f64 = prec == FEM_FP64 || prec == FEM_FP64_DF;
    carve(n_cells, n_verts, dim, f64 ? 8 : 4, work, &w, dim);
    const Operator op{1, nullptr, lam, mu};
    if (f64)
        return pcg_run<double>(dim, n_cells, n_verts, coords, conn, op, n_q, qpts, qw, node_ptr, node_idx, fixed, b, x,
                               max_iter, rtol, w, iters_out, resid_out, prec, stream);
    return pcg_run<float>(dim, n_cells, n_verts, coords, conn, op, n_q, qpts, qw, node_ptr, node_idx, fixed, b, x,
                          max_iter, rtol, w, iters_out, resid_out, prec, stream);
}

// ------------------------------------------------------------------ mixed-precision refinement
//
// fem_pcg_laplacian_refined: iterative refinement around the float32-mixed solve. Each
// outer step forms the true residual r = b - A x of the float64 iterate with the float64
// (or double-float) residual kernel, solves A d = r approximately with the PCG above in the
// FP32-mixed form (float32 values, the headline kernel as its operator), and adds d to x in
// float64. The float32 operator differs from the float64 one by ~1e-7 relative, so each
// outer step gains several digits and the iterate converges to the float64 solution; most
// of the work runs at float32 speed.

namespace fem {

__global__ void to_f32_kernel(int64_t n, const double *a, float *b) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) b[i] = static_cast<float>(a[i]);
}

// r = b - q on the free vertices, 0 on fixed ones; r32 = r rounded to float32; d32 = 0
// (N = n_comp V entries, component-major)
__global__ void refine_residual_kernel(int64_t N, int64_t V, const double *b, const double *q, const uint8_t *fixed,
                                       double *r, float *r32, float *d32) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += stride) {
        const double ri = fixed[i % V] ? 0.0 : (b ? b[i] : 0.0) - q[i];
        r[i] = ri;
        r32[i] = static_cast<float>(ri);
        d32[i] = 0.0f;
    }
}

// x += d on the free vertices
__global__ void refine_update_kernel(int64_t N, int64_t V, const uint8_t *fixed, const float *d, double *x) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += stride)
        if (!fixed[i % V]) x[i] += static_cast<double>(d[i]);
}

struct RefineWork {
    Workspace inner;    // the float32 PCG's
    float *coef32[2];   // K (Laplacian) or lambda, mu (elasticity) rounded to float32
    float *r32, *d32;
    double *elem, *q, *r, *partial, *scalars;
};

// physics 0: Laplacian (one coefficient, one component), 1: elasticity (two, dim)
static size_t carve_refined(int64_t C, int64_t V, int dim, int n_q, int physics, void *base, RefineWork *w) {
    const int nc = physics == 0 ? 1 : dim, ncoef = physics == 0 ? 1 : 2;
    Workspace inner;
    size_t off = carve(C, V, dim, sizeof(float), base, &inner, nc);
    char *b = static_cast<char *>(base);
    auto take = [&](size_t bytes) {
        void *p = b ? b + off : nullptr;
        off += align256(bytes);
        return p;
    };
    const size_t N = size_t(nc) * size_t(V);
    float *coef32[2] = {nullptr, nullptr};
    for (int c = 0; c < ncoef; ++c) coef32[c] = static_cast<float *>(take(size_t(n_q) * size_t(C) * sizeof(float)));
    float *r32 = static_cast<float *>(take(N * sizeof(float)));
    float *d32 = static_cast<float *>(take(N * sizeof(float)));
    double *elem = static_cast<double *>(take(size_t(dim + 1) * size_t(nc) * size_t(C) * sizeof(double)));
    double *q = static_cast<double *>(take(N * sizeof(double)));
    double *r = static_cast<double *>(take(N * sizeof(double)));
    double *partial = static_cast<double *>(take(sizeof(double) * kDotBlocks));
    double *scalars = static_cast<double *>(take(sizeof(double) * 2));
    if (w) *w = RefineWork{inner, {coef32[0], coef32[1]}, r32, d32, elem, q, r, partial, scalars};
    return off;
}

// the refinement loop of both entry points (arguments validated by the caller); coef64:
// K, or lambda and mu, in float64
static fem_status refined_run(int physics, int dim, int64_t C, int64_t V, const double *coords, const int32_t *conn,
                              const double *const *coef64, int n_q, const double *qpts, const double *qw,
                              const int32_t *ptr, const int32_t *idx, const uint8_t *fixed, const double *b,
                              double *x, int max_outer, int max_inner, double inner_rtol, double rtol,
                              const RefineWork &w, int *outer_out, int *inner_out, double *resid_out,
                              fem_precision residual_prec, cudaStream_t stream) {
    const int nc = physics == 0 ? 1 : dim, ncoef = physics == 0 ? 1 : 2;
    const int64_t N = int64_t(nc) * V;
    const int gV = static_cast<int>(std::min<int64_t>((N + 255) / 256, 4096));
    const int gK = static_cast<int>(std::min<int64_t>((int64_t(n_q) * C + 255) / 256, 4096));
    for (int c = 0; c < ncoef; ++c) to_f32_kernel<<<gK, 256, 0, stream>>>(int64_t(n_q) * C, coef64[c], w.coef32[c]);
    fem_status st = check_launch("refined solve");
    if (st != FEM_OK) return st;
    const Operator op32 = physics == 0 ? Operator{0, w.coef32[0], nullptr, nullptr}
                                       : Operator{1, nullptr, w.coef32[0], w.coef32[1]};
    double rn0 = 0.0, rn = 0.0;
    int outer = 0, inner_total = 0;
    for (;;) {
        // the true residual of the float64 iterate
        st = physics == 0 ? fem_integrate_laplacian(dim, C, V, coords, conn, x, coef64[0], n_q, qpts, qw, w.elem,
                                                    residual_prec, stream)
                          : fem_integrate_elasticity(dim, C, V, coords, conn, x, coef64[0], coef64[1], n_q, qpts, qw,
                                                     w.elem, residual_prec, stream);
        if (st != FEM_OK) return st;
        if ((st = launch_gather(dim, nc, C, V, w.elem, ptr, idx, w.q, FEM_FP64, stream)) != FEM_OK) return st;
        refine_residual_kernel<<<gV, 256, 0, stream>>>(N, V, b, w.q, fixed, w.r, w.r32, w.d32);
        dot_partial_kernel<double><<<kDotBlocks, 256, 0, stream>>>(N, w.r, w.r, w.partial);
        dot_final_kernel<<<1, 256, 0, stream>>>(w.partial, w.scalars);
        double rr = 0.0;
        cudaError_t e = cudaMemcpyAsync(&rr, w.scalars, sizeof(double), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return fail(FEM_ERR_CUDA, "refined solve: %s", cudaGetErrorString(e));
        rn = std::sqrt(rr);
        if (outer == 0) rn0 = rn;
        if (rn <= rtol * rn0 || rn == 0.0 || outer >= max_outer) break;
        // the correction in the FP32-mixed form: A d = r, d = 0 on the fixed vertices. When
        // the reduction still needed is less than one correction at inner_rtol gives, and
        // within float32's reach, the last correction is solved to a third of it instead, so
        // that it ends the refinement rather than stopping just short of rtol.
        const double need = rtol * rn0 / rn;
        const double tol_k = (0.3 * need < inner_rtol && 0.3 * need >= 1e-6) ? 0.3 * need : inner_rtol;
        int it = 0;
        double res = 0.0;
        st = pcg_run<float>(dim, C, V, coords, conn, op32, n_q, qpts, qw, ptr, idx, fixed, w.r32, w.d32, max_inner,
                            tol_k, w.inner, &it, &res, FEM_FP32_MIXED, stream, outer > 0);
        if (st != FEM_OK) return st;
        inner_total += it;
        refine_update_kernel<<<gV, 256, 0, stream>>>(N, V, fixed, w.d32, x);
        if ((st = check_launch("refined solve")) != FEM_OK) return st;
        ++outer;
    }
    if (outer_out) *outer_out = outer;
    if (inner_out) *inner_out = inner_total;
    if (resid_out) *resid_out = rn0 > 0.0 ? rn / rn0 : 0.0;
    return check_launch("refined solve");
}

// the argument checks both entry points share
static fem_status refined_check(int dim, int64_t C, int64_t V, const double *coords, const int32_t *conn, int n_q,
                                int max_outer, int max_inner, double inner_rtol, double rtol,
                                fem_precision residual_prec, int *outer_out, int *inner_out, double *resid_out) {
    fem_status st = check_common(dim, C, V, coords, conn);
    if (st != FEM_OK) return st;
    if (residual_prec != FEM_FP64 && residual_prec != FEM_FP64_DF)
        return fail(FEM_ERR_ARG, "residual_prec must be FEM_FP64 or FEM_FP64_DF");
    if (max_outer < 0 || max_inner < 0 || !(rtol >= 0.0) || !(inner_rtol > 0.0 && inner_rtol < 1.0))
        return fail(FEM_ERR_ARG, "max_outer, max_inner must be >= 0, rtol >= 0 and 0 < inner_rtol < 1");
    if (n_q < 1 || n_q > FEM_MAX_QPTS) return fail(FEM_ERR_SHAPE, "n_q = %d outside [1, %d]", n_q, FEM_MAX_QPTS);
    if (outer_out) *outer_out = 0;
    if (inner_out) *inner_out = 0;
    if (resid_out) *resid_out = 0.0;
    return FEM_OK;
}

}  // namespace fem

extern "C" int64_t fem_pcg_refined_work_bytes(int dim, int64_t n_cells, int64_t n_verts, int n_q) {
    if ((dim != 2 && dim != 3) || n_cells < 0 || n_verts < 0 || n_q < 1 || n_q > FEM_MAX_QPTS) return -1;
    return static_cast<int64_t>(carve_refined(n_cells, n_verts, dim, n_q, 0, nullptr, nullptr));
}

extern "C" int64_t fem_pcg_elasticity_refined_work_bytes(int dim, int64_t n_cells, int64_t n_verts, int n_q) {
    if ((dim != 2 && dim != 3) || n_cells < 0 || n_verts < 0 || n_q < 1 || n_q > FEM_MAX_QPTS) return -1;
    return static_cast<int64_t>(carve_refined(n_cells, n_verts, dim, n_q, 1, nullptr, nullptr));
}

extern "C" fem_status fem_pcg_laplacian_refined(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                                const int32_t *conn, const double *K, int n_q, const double *qpts,
                                                const double *qw, const int32_t *node_ptr, const int32_t *node_idx,
                                                const uint8_t *fixed, const double *b, double *x, int max_outer,
                                                int max_inner, double inner_rtol, double rtol, void *work,
                                                int64_t work_bytes, int *outer_out, int *inner_out,
                                                double *resid_out, fem_precision residual_prec, fem_stream stream) {
    fem_status st = refined_check(dim, n_cells, n_verts, coords, conn, n_q, max_outer, max_inner, inner_rtol, rtol,
                                  residual_prec, outer_out, inner_out, resid_out);
    if (st != FEM_OK || n_verts == 0) return st;
    if (!K || !node_ptr || !node_idx || !fixed || !x || !work) return fail(FEM_ERR_ARG, "a NULL array argument");
    const int64_t need = fem_pcg_refined_work_bytes(dim, n_cells, n_verts, n_q);
    if (work_bytes < need)
        return fail(FEM_ERR_OOM, "fem_pcg_laplacian_refined: workspace of %lld bytes, %lld needed",
                    static_cast<long long>(work_bytes), static_cast<long long>(need));
    if (reinterpret_cast<uintptr_t>(work) & 255u) return fail(FEM_ERR_ARG, "work must be 256-byte aligned");
    RefineWork w;
    carve_refined(n_cells, n_verts, dim, n_q, 0, work, &w);
    const double *coef[1] = {K};
    return refined_run(0, dim, n_cells, n_verts, coords, conn, coef, n_q, qpts, qw, node_ptr, node_idx, fixed, b, x,
                       max_outer, max_inner, inner_rtol, rtol, w, outer_out, inner_out, resid_out, residual_prec,
                       stream);
}

extern "C" fem_status fem_pcg_elasticity_refined(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                                 const int32_t *conn, const double *lam, const double *mu, int n_q,
                                                 const double *qpts, const double *qw, const int32_t *node_ptr,
                                                 const int32_t *node_idx, const uint8_t *fixed, const double *b,
                                                 double *x, int max_outer, int max_inner, double inner_rtol,
                                                 double rtol, void *work, int64_t work_bytes, int *outer_out,
                                                 int *inner_out, double *resid_out, fem_precision residual_prec,
                                                 fem_stream stream) {
    fem_status st = refined_check(dim, n_cells, n_verts, coords, conn, n_q, max_outer, max_inner, inner_rtol, rtol,
                                  residual_prec, outer_out, inner_out, resid_out);
    if (st != FEM_OK || n_verts == 0) return st;
    if (int64_t(dim) * n_verts >= (int64_t(1) << 31)) return fail(FEM_ERR_SHAPE, "too many vertices");
    if (!lam || !mu || !node_ptr || !node_idx || !fixed || !x || !work)
        return fail(FEM_ERR_ARG, "a NULL array argument");
    const int64_t need = fem_pcg_elasticity_refined_work_bytes(dim, n_cells, n_verts, n_q);
    if (work_bytes < need)
        return fail(FEM_ERR_OOM, "fem_pcg_elasticity_refined: workspace of %lld bytes, %lld needed",
                    static_cast<long long>(work_bytes), static_cast<long long>(need));
    if (reinterpret_cast<uintptr_t>(work) & 255u) return fail(FEM_ERR_ARG, "work must be 256-byte aligned");
    RefineWork w;
    carve_refined(n_cells, n_verts, dim, n_q, 1, work, &w);
    const double *coef[2] = {lam, mu};
    return refined_run(1, dim, n_cells, n_verts, coords, conn, coef, n_q, qpts, qw, node_ptr, node_idx, fixed, b, x,
                       max_outer, max_inner, inner_rtol, rtol, w, outer_out, inner_out, resid_out, residual_prec,
                       stream);
}
