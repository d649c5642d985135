/*
 * fem.h -- C ABI of libfem: batched quadrature-based P1 element integration on GB300.
 *
 * Method: Knepley, Rupp, Terrel, "Finite Element Integration with Quadrature on the
 * GPU". For every cell of a simplex mesh the library evaluates the bracket of Eq. 2
 * with f0 = 0,
 *
 *     r_{e,b} = sum_q w_q |det J_e| (J_e^{-T} grad_ref phi_b(xi_q)) . f1(u, grad u)(x_q),
 *
 * producing unassembled per-cell element vectors. The pointwise functions are the
 * two of Sec. 6: the variable-coefficient Laplacian f1 = K grad u (Sec. 2) and linear
 * elasticity, generalised from the paper's symmetric-gradient listing to the Lame
 * stress f1 = lambda tr(eps) I + 2 mu eps, eps = (grad u + grad u^T)/2.
 * The affine Jacobian J = [x_1 - x_0 | ... | x_d - x_0], its determinant and its
 * inverse are computed in-kernel from the vertex coordinates (the paper loads them
 * precomputed, Sec. 3 and Appendix).
 *
 * Conventions shared by every entry point:
 *  - All array arguments are DEVICE pointers owned by the caller, except qpts and qw,
 *    which are small HOST tables copied into the launch (and the host arrays of
 *    fem_integrate_laplacian_host). No entry point allocates device memory for data or
 *    synchronises the stream: work is enqueued on `stream` (0 = the legacy default
 *    stream) and the call returns after the launch. The one exception is
 *    fem_pcg_laplacian, which waits for its result and runs its loop as a CUDA graph.
 *  - Outside stream capture the integration, adjoint, geometry and assembly kernels are
 *    launched with programmatic stream serialisation (programmatic dependent launch):
 *    a kernel may be scheduled onto the GPU while the kernel before it on `stream`
 *    drains, and waits, before touching memory, until that kernel has completed and its
 *    writes are visible. Stream order for data is unchanged; only the launch gap goes.
 *    Under capture the launches are plain.
 *  - Layouts are structure-of-arrays with the cell (or vertex) index fastest:
 *        coords [dim][n_verts]        always float64
 *        conn   [dim+1][n_cells]      int32 vertex ids in [0, n_verts)
 *        u      [n_verts] (Laplacian) or [dim][n_verts] (elasticity)
 *        K, lam, mu [n_q][n_cells]    one coefficient per quadrature point
 *        out    [(dim+1)*n_comp][n_cells], row b*n_comp + k (n_comp = 1 or dim)
 *    Value arrays (u, K, lam, mu, out, lambda, dK, du, scratch) are float64 for
 *    FEM_FP64 and FEM_FP64_DF and float32 for FEM_FP32_MIXED and FEM_FP32.
 *  - Reference simplex: vertices 0, e_1, ..., e_d. qpts [n_q][dim] are reference
 *    coordinates and qw [n_q] the weights (they sum to 1/d! for an exact rule).
 *    The P1 reference gradients are constant, so only the weights enter the
 *    arithmetic; qpts may be NULL and, when given, must lie in the reference simplex.
 *  - Errors are returned synchronously (argument checks, launch failures); an error
 *    leaves the outputs untouched or partially written. fem_last_error() gives a
 *    thread-local message for the most recent failing call. No exception crosses
 *    the ABI. n_cells = 0 is a valid no-op.
 *  - Vertex ids are clamped into [0, n_verts) in-kernel, so malformed connectivity
 *    cannot make a kernel read out of bounds; it gives meaningless values for the cells
 *    concerned instead. Every kernel also checks its mesh as it goes (the mesh check of
 *    the boundary, always on): a vertex id outside [0, n_verts), or a cell with det J = 0
 *    or a non-finite det J, or with a repeated vertex id, sets a bit in the device error
 *    word, and the next fem_device_error() returns FEM_ERR_BADMESH. (The mixed form
 *    checks the determinant of the cells its shape test sends to float64, which every
 *    degenerate cell fails for tau > 0.) fem_check_mesh() counts such cells.
 *  - Vectorised (128-bit) loads are used when every cell-indexed row is 16-byte
 *    aligned (n_cells a multiple of 4 and 16-byte aligned base pointers); other
 *    inputs run the same kernels with scalar loads, still on the GPU.
 */
#ifndef FEM_H
#define FEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *fem_stream; /* identical to cudaStream_t */

typedef enum {
    FEM_OK = 0,
    FEM_ERR_ARG = -1,       /* bad scalar argument or NULL pointer */
    FEM_ERR_SHAPE = -2,     /* sizes out of the supported range */
    FEM_ERR_CUDA = -3,      /* a CUDA launch or runtime call failed */
    FEM_ERR_OOM = -4,       /* a caller-provided buffer is too small */
    FEM_ERR_BADMESH = -5,   /* fem_device_error: a kernel met an invalid mesh */
    FEM_ERR_TIMEOUT = -6,   /* a bounded device-side wait gave up */
    FEM_ERR_UNSUPPORTED = -7
} fem_status;

typedef enum {
    /* every value and every operation in float64 (the reciprocal of |det J| starts from a
     * float32 seed refined by two float64 Newton steps: within about an ulp of the IEEE
     * quotient) */
    FEM_FP64 = 0,
    /* values stored in float32; coordinates read as float64 and split into float32
     * (hi, lo) pairs so the Jacobian columns are exact to float32 rounding; geometry
     * and physics in float32; the quadrature sum of the element vector compensated
     * (TwoSum/TwoProduct); cells failing the shape test |det J| >= tau prod_j |J e_j|
     * (Hadamard ratio) or giving a non-finite result are recomputed in float64 */
    FEM_FP32_MIXED = 1,
    /* ablation: float32 values, coordinates rounded to float32 before the Jacobian,
     * plain float32 sums, no float64 fallback */
    FEM_FP32 = 2,
    /* float64 values (as FEM_FP64) with float64-class accuracy computed on the float32
     * pipe: the Jacobian columns are formed in float64, every other intermediate is a
     * pair of float32 values (hi + lo, double-length arithmetic from TwoSum/TwoProduct),
     * the outputs are widened back to float64. Values must lie in float32's normal range
     * (|x| in [2^-126, 2^128), or zero). fem_integrate_laplacian, fem_integrate_elasticity,
     * fem_adjoint_laplacian (its element part; the vertex sum in float64), (for its
     * residual) fem_pcg_laplacian, and fem_gather_nodes (float64 sums) only; the other
     * entry points return FEM_ERR_ARG for it. */
    FEM_FP64_DF = 3
} fem_precision;

#define FEM_MAX_QPTS 32

/* ---------------------------------------------------------------------------------
 * fem_integrate_laplacian -- element residuals of the variable-coefficient Laplacian
 * (Eq. 2 with f0 = 0, f1 = K grad u; Sec. 2 and the Sec. 6 Laplacian listing).
 *   dim        2 (triangles) or 3 (tetrahedra)
 *   n_cells    C >= 0, n_verts V >= 1 (when C > 0); (dim+1)*C and V below 2^31
 *   coords     [dim][V] float64
 *   conn       [dim+1][C] int32
 *   u          [V] nodal values
 *   K          [n_q][C] coefficient at each quadrature point of each cell
 *   n_q        1..FEM_MAX_QPTS; qpts [n_q][dim] (host, may be NULL), qw [n_q] (host)
 *   elem_out   [dim+1][C] element vectors (written)
 * Returns FEM_OK, FEM_ERR_ARG, FEM_ERR_SHAPE or FEM_ERR_CUDA.
 * ------------------------------------------------------------------------------- */
fem_status fem_integrate_laplacian(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                   const int32_t *conn, const void *u, const void *K, int n_q,
                                   const double *qpts, const double *qw, void *elem_out,
                                   fem_precision prec, fem_stream stream);

/* ---------------------------------------------------------------------------------
 * fem_integrate_laplacian_fields -- fem_integrate_laplacian for n_fields nodal fields on
 * the same mesh and coefficient (Eq. 2 with f1 = K grad u, once per field): the geometry
 * of each cell (coordinate gathers, J, det J, adjugate) and Kbar / |det J| are computed
 * once and reused for every field, so each extra field costs its nodal gathers, the
 * contraction and its element-vector stores.
 *   u          [n_fields][n_verts] nodal values, field-major
 *   elem_out   [n_fields][dim+1][n_cells] element vectors (written)
 * Other arguments, precisions (not FEM_FP64_DF) and returns as fem_integrate_laplacian;
 * n_fields = 0 is a no-op. Per field and cell the arithmetic is that of the single-field
 * per-cell kernel, so results equal fem_integrate_laplacian's bit for bit in FEM_FP64
 * (and in the float32 forms when that call takes its per-cell path).
 * ------------------------------------------------------------------------------- */
fem_status fem_integrate_laplacian_fields(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                          const int32_t *conn, int n_fields, const void *u, const void *K,
                                          int n_q, const double *qpts, const double *qw, void *elem_out,
                                          fem_precision prec, fem_stream stream);

/* ---------------------------------------------------------------------------------
 * fem_integrate_elasticity -- element residuals of linear elasticity (Eq. 2 with f0 = 0
 * and the vector form of Eq. 1: f1 = lambda tr(eps) I + 2 mu eps; with lambda = 0,
 * mu = 1/2 this is the Sec. 6 elasticity listing).
 *   u          [dim][V] nodal displacement components
 *   lam, mu    [n_q][C] Lame parameters at each quadrature point
 *   elem_out   [(dim+1)*dim][C], row b*dim + k = component k of basis function b
 * Other arguments and returns as fem_integrate_laplacian.
 * ------------------------------------------------------------------------------- */
fem_status fem_integrate_elasticity(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                    const int32_t *conn, const void *u, const void *lam, const void *mu,
                                    int n_q, const double *qpts, const double *qw, void *elem_out,
                                    fem_precision prec, fem_stream stream);

/* ---------------------------------------------------------------------------------
 * fem_integrate_reaction_diffusion -- element vectors of the full bracket of Eq. 2 (both
 * the f0 and the f1 term) with pointwise functions that take an auxiliary field a and
 * its gradient (Eq. 8; Sec. 4 allows a in the space of u or in P0):
 *     f1 = a grad u,  f0 = c u + drift grad a . grad u,
 *     r_b = sum_q w_q |det J| [ phi_b(xi_q) f0(xi_q) + G_b . a(xi_q) grad u ]
 *   u          [V] nodal values
 *   a          a_space = 1: [V] nodal values of a P1 field, a(xi_q) = sum_b phi_b(xi_q) a_b
 *              a_space = 0: [C] one value per cell (P0; grad a = 0 inside a cell)
 *   c          [n_q][C] reaction coefficient per quadrature point, or NULL (no c u term)
 *   drift      scalar g of the first-order term along grad a (0: none; must be finite)
 *   qpts       required here (phi_b(xi_q) enters both terms)
 *   elem_out   [dim+1][C]
 * Other arguments and returns as fem_integrate_laplacian. The FP32_MIXED form computes
 * sum_q w_q a(xi_q) with the compensated sum and recomputes badly shaped cells in
 * float64; the f0 sum is a plain float32 sum.
 * ------------------------------------------------------------------------------- */
fem_status fem_integrate_reaction_diffusion(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                            const int32_t *conn, const void *u, const void *a, int a_space,
                                            const void *c, double drift, int n_q, const double *qpts,
                                            const double *qw, void *elem_out, fem_precision prec,
                                            fem_stream stream);

/* ---------------------------------------------------------------------------------
 * fem_integrate_pointwise -- element vectors of the full bracket of Eq. 2 for pointwise
 * functions f0 and f1 given as CUDA C++ source text, compiled at run time (Sec. 5: the
 * library user provides f0 and f1 as strings, which are inlined into the kernel source
 * handed to the just-in-time compiler). For a field of n_comp components:
 *     r_{e,b,k} = sum_q w_q |det J| [ phi_b(xi_q) f0_k(q) + sum_i G_{b,i} f1_{k,i}(q) ]
 * with G_b = J^{-T} grad_ref phi_b and, at every quadrature point, the field, its gradient,
 * the coefficients and the physical point.
 *   f0_src, f1_src  function BODIES (either may be NULL = zero; not both). In scope:
 *                   const T *u       [NCOMP]        u_k(q) = sum_b phi_b(xi_q) u_{b,k}
 *                   const T *grad_u  [NCOMP*DIM]    grad_u[k*DIM + i] = d u_k / d x_i
 *                   const T *a       [NCOEF]        a[j] = coef[j][q][e]
 *                   const T *x       [DIM]          x(q) = sum_b phi_b(xi_q) x_b
 *                   T *f0 [NCOMP] or T *f1 [NCOMP*DIM] (zeroed before the call), to fill
 *                   and the constants DIM, NCOMP, NCOEF; T is double (FEM_FP64) or float
 *                   (FEM_FP32_MIXED). Example, the variable-coefficient Laplacian:
 *                     f1_src = "for (int i = 0; i < DIM; ++i) f1[i] = a[0] * grad_u[i];"
 *   n_comp          1..3 field components; u is [n_comp][n_verts]
 *   n_coef          0..FEM_POINTWISE_MAX_COEF per-point coefficients; coef [n_coef][n_q][n_cells]
 *   qpts            required (phi_b(xi_q) enters u(q), x(q) and the f0 term)
 *   elem_out        [(dim+1)*n_comp][n_cells], row b*n_comp + k
 *   prec            FEM_FP64 (all float64) or FEM_FP32_MIXED (values, physics and sums in
 *                   float32; coordinates split exactly into float32 pairs for the Jacobian;
 *                   cells failing the shape test get their geometry in float64)
 * The first call for a given (device, precision, dim, n_comp, n_coef, n_q, f0_src, f1_src)
 * compiles the kernel with NVRTC for the device's architecture and loads it (tens to
 * hundreds of milliseconds); later calls reuse the cached kernel. A call with n_cells = 0
 * compiles and caches without launching: make it before any stream capture, which must
 * not contain a compilation. Returns FEM_ERR_ARG with the compiler's log in
 * fem_last_error() when the source does not compile, FEM_ERR_UNSUPPORTED when NVRTC
 * (libnvrtc.so) cannot be loaded; otherwise as fem_integrate_laplacian. Mesh errors are
 * reported through fem_device_error() like the built-in kernels.
 * ------------------------------------------------------------------------------- */
#define FEM_POINTWISE_MAX_COEF 8
fem_status fem_integrate_pointwise(const char *f0_src, const char *f1_src, int dim, int n_comp, int n_coef,
                                   int64_t n_cells, int64_t n_verts, const double *coords, const int32_t *conn,
                                   const void *u, const void *coef, int n_q, const double *qpts, const double *qw,
                                   void *elem_out, fem_precision prec, fem_stream stream);

/* ---------------------------------------------------------------------------------
 * fem_integrate_laplacian_host -- fem_integrate_laplacian for arrays in HOST memory
 * (coords_h, conn_h, u_h, K_h in, out_h [dim+1][C] out; same layouts). The vertex arrays
 * are copied to the device once. Then, with chunks >= 1, the cells are processed in
 * `chunks` pieces on two library-owned streams, so that uploads, kernels and downloads of
 * different chunks overlap; with chunks == 0 nothing more is copied: the kernel reads
 * conn_h and K_h and writes out_h directly across the host link (these three must then be
 * page-locked and device-mapped, e.g. cudaHostAlloc / pinned tensors; otherwise
 * FEM_ERR_ARG). All device buffers come from `work` (fem_host_work_bytes() bytes for the
 * same `chunks`, 256-byte aligned, caller-owned); nothing is allocated. With chunks >= 1
 * the host arrays should be page-locked for the copies to be asynchronous; pageable
 * memory works but the copies then serialise. The call returns after enqueueing; the
 * results are in out_h once `stream` has completed. Calls from several host threads on
 * one device must be serialised by the caller (the library's two streams and events are
 * shared). FEM_FP64, FEM_FP32_MIXED and FEM_FP32 only.
 * ------------------------------------------------------------------------------- */
int64_t fem_host_work_bytes(int dim, int64_t n_cells, int64_t n_verts, int n_q, fem_precision prec, int chunks);
fem_status fem_integrate_laplacian_host(int dim, int64_t n_cells, int64_t n_verts, const double *coords_h,
                                        const int32_t *conn_h, const void *u_h, const void *K_h, int n_q,
                                        const double *qpts, const double *qw, void *out_h, void *work,
                                        int64_t work_bytes, int chunks, fem_precision prec, fem_stream stream);

/* ---------------------------------------------------------------------------------
 * The paper's thread-transposition kernel (Sec. 3, Figs. 1-3), rebuilt as an ablation:
 *
 * fem_element_values -- the closure of a nodal field: ue[b][e] = u[conn[b][e]], [dim+1][C]
 *   (the element-local basis coefficients the paper's kernel reads).
 * fem_integrate_laplacian_transposed -- the Laplacian element residual from ue, K and the
 *   geometry of fem_precompute_geometry, computed the paper's way: per batch of
 *   cells_per_batch cells (32, 64, 128; 256 in the float32 forms) the inputs go to shared
 *   memory, one thread per (cell, quadrature point) evaluates f1 (Sec. 3.1), a barrier,
 *   one thread per (cell, basis function) contracts (Sec. 3.2); a thread block runs
 *   batches_per_block batches in turn. Requires n_q = dim + 1 (= N_b, as in the rules
 *   used here). Value type float64 for FEM_FP64, float32 otherwise (no compensation).
 * Results equal fem_integrate_laplacian's up to rounding; this path exists to measure
 * the paper's design on GB300 (Table 2 analogue: a sweep over both batch parameters).
 * ------------------------------------------------------------------------------- */
fem_status fem_element_values(int dim, int64_t n_cells, int64_t n_verts, const int32_t *conn, const void *u,
                              void *ue, fem_precision prec, fem_stream stream);
fem_status fem_integrate_laplacian_transposed(int dim, int64_t n_cells, const void *ue, const void *K, int n_q,
                                              const double *qpts, const double *qw, const void *geom,
                                              void *elem_out, int cells_per_batch, int batches_per_block,
                                              fem_precision prec, fem_stream stream);

/* ---------------------------------------------------------------------------------
 * fem_pcg_laplacian -- solve A x = b with a matrix-free Jacobi-preconditioned conjugate
 * gradient, A the assembled operator of Eq. 2 for the variable-coefficient Laplacian
 * (element residuals of fem_integrate_laplacian summed per vertex, E^T r_e(x)), not in
 * the paper. Vertices with fixed[v] != 0 are Dirichlet vertices: they keep the value
 * that x holds on entry, and the system is solved on the other vertices.
 *   K, n_q, qpts, qw, coords, conn   as fem_integrate_laplacian
 *   node_ptr, node_idx   from fem_build_node2cell for conn
 *   fixed      [V] uint8 Dirichlet mask
 *   b          [V] right-hand side (load vector), or NULL for zero
 *   x          [V] in: initial guess and Dirichlet values; out: the solution
 *   max_iter, rtol       stop when ||r||_2 <= rtol ||r_0||_2 or after max_iter iterations
 *   work       caller-owned device workspace of fem_pcg_work_bytes() bytes, 256-byte aligned
 *   iters_out, resid_out (host, may be NULL) iterations taken and ||r|| / ||r_0||
 * Value arrays are float64 for FEM_FP64 and FEM_FP64_DF (the residual then runs in the
 * double-float form: float64-class accuracy at float32-pipe speed) and float32 otherwise;
 * dot products accumulate in float64 in a fixed order (reproducible). The iteration is CG
 * in Chronopoulos and Gear's form (both inner products of an iteration from one reduction:
 * 3 kernels per iteration). The iterations run on the device as a CUDA graph with a WHILE
 * node (one iteration captured as its body, the condition set by the body's last kernel),
 * so the host does not wait per iteration;
 * unlike the other entry points this one returns only after the solve: it synchronises
 * `stream` twice (initial residual norm, final iteration count). The loop body is
 * captured on a library-owned stream per device, one capture at a time (a lock), so
 * calls from several host threads are safe.
 * ------------------------------------------------------------------------------- */
int64_t fem_pcg_work_bytes(int dim, int64_t n_cells, int64_t n_verts, fem_precision prec);
fem_status fem_pcg_laplacian(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                             const int32_t *conn, const void *K, int n_q, const double *qpts, const double *qw,
                             const int32_t *node_ptr, const int32_t *node_idx, const uint8_t *fixed,
                             const void *b, void *x, int max_iter, double rtol, void *work, int64_t work_bytes,
                             int *iters_out, double *resid_out, fem_precision prec, fem_stream stream);

/* ---------------------------------------------------------------------------------
 * fem_pcg_elasticity -- the same Jacobi-PCG for linear elasticity (not in the paper): A the
 * assembled operator of fem_integrate_elasticity (element residuals summed per vertex and
 * component), unknowns u [dim][V] (component-major, as fem_integrate_elasticity's u), the
 * Jacobi diagonal from the element stiffness diagonals. A vertex with fixed[v] != 0 keeps
 * all dim components of x. lam, mu [n_q][C]; b, x [dim][V]; the rest as fem_pcg_laplacian,
 * with a workspace of fem_pcg_elasticity_work_bytes() bytes.
 * ------------------------------------------------------------------------------- */
int64_t fem_pcg_elasticity_work_bytes(int dim, int64_t n_cells, int64_t n_verts, fem_precision prec);
fem_status fem_pcg_elasticity(int dim, int64_t n_cells, int64_t n_verts, const double *coords, const int32_t *conn,
                              const void *lam, const void *mu, int n_q, const double *qpts, const double *qw,
                              const int32_t *node_ptr, const int32_t *node_idx, const uint8_t *fixed, const void *b,
                              void *x, int max_iter, double rtol, void *work, int64_t work_bytes, int *iters_out,
                              double *resid_out, fem_precision prec, fem_stream stream);

/* ---------------------------------------------------------------------------------
 * fem_pcg_laplacian_refined -- the same system solved by mixed-precision iterative
 * refinement (not in the paper): each outer step forms the true residual r = b - A x of
 * the float64 iterate with the residual kernel in residual_prec (FEM_FP64 or FEM_FP64_DF),
 * solves A d = r with fem_pcg_laplacian's Jacobi-PCG in FEM_FP32_MIXED (float32 values,
 * K rounded to float32 once, to relative residual inner_rtol or max_inner iterations; a
 * correction that only has to gain the last factor f < inner_rtol / 0.3 of the reduction,
 * with 0.3 f >= 1e-6, is solved to 0.3 f instead) and sets x += d in float64 on the free
 * vertices. It stops when ||r|| <= rtol ||r_0|| (r_0 the
 * residual of the initial x, both in float64) or after max_outer corrections.
 *   K, b, x    float64 ([n_q][C], [V] or NULL, [V]: initial guess and Dirichlet values in,
 *              solution out); the other arguments as fem_pcg_laplacian
 *   work       caller-owned device workspace of fem_pcg_refined_work_bytes() bytes, 256-byte
 *              aligned (holds the float32 solve's workspace, K in float32, the float64 residual)
 *   outer_out, inner_out, resid_out (host, may be NULL): corrections made, float32 PCG
 *              iterations in all, ||r|| / ||r_0|| of the returned x
 * Synchronises `stream` once per outer step (the residual norm) and as fem_pcg_laplacian
 * does inside each correction; returns when the solve has finished.
 * ------------------------------------------------------------------------------- */
int64_t fem_pcg_refined_work_bytes(int dim, int64_t n_cells, int64_t n_verts, int n_q);
int64_t fem_pcg_elasticity_refined_work_bytes(int dim, int64_t n_cells, int64_t n_verts, int n_q);
fem_status fem_pcg_laplacian_refined(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                     const int32_t *conn, const double *K, int n_q, const double *qpts,
                                     const double *qw, const int32_t *node_ptr, const int32_t *node_idx,
                                     const uint8_t *fixed, const double *b, double *x, int max_outer, int max_inner,
                                     double inner_rtol, double rtol, void *work, int64_t work_bytes, int *outer_out,
                                     int *inner_out, double *resid_out, fem_precision residual_prec,
                                     fem_stream stream);
/* fem_pcg_elasticity_refined -- the same refinement for linear elasticity (fem_pcg_elasticity's
 * operator): lam, mu [n_q][C], b, x [dim][V] in float64, both rounded to float32 once for the
 * corrections; workspace of fem_pcg_elasticity_refined_work_bytes() bytes. */
fem_status fem_pcg_elasticity_refined(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                      const int32_t *conn, const double *lam, const double *mu, int n_q,
                                      const double *qpts, const double *qw, const int32_t *node_ptr,
                                      const int32_t *node_idx, const uint8_t *fixed, const double *b, double *x,
                                      int max_outer, int max_inner, double inner_rtol, double rtol, void *work,
                                      int64_t work_bytes, int *outer_out, int *inner_out, double *resid_out,
                                      fem_precision residual_prec, fem_stream stream);

/* ---------------------------------------------------------------------------------
 * The paper's precomputed-geometry layout (Sec. 3 and the Appendix load J^{-1} and det J
 * per cell rather than computing them), as an alternate entry for the Laplacian:
 *
 * fem_precompute_geometry -- per-mesh pass writing geom [dim*dim + 1][C] in the value
 *   type of prec: rows i*dim + j hold (J^{-1})_{ij} (row-major), row dim*dim holds det J
 *   (signed). Computed in float64, rounded once to float32 for the float32 forms.
 * fem_integrate_laplacian_geom -- the Laplacian element residual of
 *   fem_integrate_laplacian from conn, u, K and that geom (no coordinates):
 *   r_b = (sum_q w_q K_q) |det J| G_b . g, G_b = J^{-T} grad_ref phi_b, g = sum_b u_b G_b.
 *   Both float32 forms integrate float32 geometry (FEM_FP32_MIXED keeps its compensated
 *   quadrature sum; there is no float64 recomputation without coordinates).
 * Arguments otherwise as fem_integrate_laplacian; geom is a caller-owned device array.
 * ------------------------------------------------------------------------------- */
fem_status fem_precompute_geometry(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                   const int32_t *conn, void *geom, fem_precision prec, fem_stream stream);
fem_status fem_integrate_laplacian_geom(int dim, int64_t n_cells, int64_t n_verts, const int32_t *conn,
                                        const void *u, const void *K, int n_q, const double *qpts,
                                        const double *qw, const void *geom, void *elem_out,
                                        fem_precision prec, fem_stream stream);

/* ---------------------------------------------------------------------------------
 * Prepared vertex records for the mixed-form Laplacian (not in the paper; the per-mesh
 * counterpart of the paper's precomputed geometry, for meshes evaluated many times):
 *
 * fem_prepare_vertices -- once per mesh: every float64 coordinate split into the float32
 *   (hi, lo) pair the mixed form differences its Jacobian columns from, written to rec,
 *   fem_prepared_record_floats(dim) floats per vertex (3D: 8 = hi_x hi_y hi_z lo_x lo_y lo_z
 *   and two unused; 2D: 4 = hi_x hi_y lo_x lo_y). rec is a caller-owned float32 device
 *   array of n_verts * fem_prepared_record_floats(dim) entries, 32-byte aligned.
 * fem_integrate_laplacian_prepared -- fem_integrate_laplacian in FEM_FP32_MIXED with the
 *   coordinate gathers and splits replaced by one record load per vertex; the element
 *   vectors are bitwise those of fem_integrate_laplacian (same operations on the same
 *   pairs). coords is still read, for the float64 recomputation of badly shaped cells.
 *   Needs an even n_cells and 8-byte aligned conn, K and elem_out (FEM_ERR_SHAPE
 *   otherwise). Other arguments as fem_integrate_laplacian (values float32).
 * ------------------------------------------------------------------------------- */
int64_t fem_prepared_record_floats(int dim);
fem_status fem_prepare_vertices(int dim, int64_t n_verts, const double *coords, float *rec, fem_stream stream);
fem_status fem_integrate_laplacian_prepared(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                            const float *rec, const int32_t *conn, const void *u, const void *K,
                                            int n_q, const double *qpts, const double *qw, void *elem_out,
                                            fem_stream stream);

/* ---------------------------------------------------------------------------------
 * fem_set_mixed_threshold / fem_get_mixed_threshold -- the shape-test threshold tau of
 * FEM_FP32_MIXED (default 0.05). tau = 0 sends no cell to the float64 path, tau > 1
 * sends every cell. Process-wide; set it between calls, not during them.
 * ------------------------------------------------------------------------------- */
fem_status fem_set_mixed_threshold(double tau);
double fem_get_mixed_threshold(void);

/* ---------------------------------------------------------------------------------
 * fem_check_mesh -- validation pass (not on the hot path). Writes into the DEVICE
 * array counts[4] (int64, overwritten):
 *   counts[0] = number of connectivity entries outside [0, V)
 *   counts[1] = number of degenerate cells: |det J| <= 16 eps_64 prod_j |J e_j| or non-finite
 *   counts[2] = number of cells FEM_FP32_MIXED sends to its float64 path
 *   counts[3] = number of non-degenerate cells with det J < 0 (inverted; allowed, |det J| is used)
 * Read counts after synchronising the stream.
 * ------------------------------------------------------------------------------- */
fem_status fem_check_mesh(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                          const int32_t *conn, int64_t *counts, fem_stream stream);

/* ---------------------------------------------------------------------------------
 * fem_adjoint_laplacian -- gradient of the scalar J(u, K) = sum_e sum_b lambda_{e,b} r_{e,b}
 * with r the Laplacian element residual above (not in the paper):
 *   dK[q][e] = dJ/dK_{e,q} = w_q |det J_e| (sum_b lambda_{e,b} G_b) . grad u_e
 *   du[n]    = dJ/du_n = sum over (e, a) with conn[a][e] = n of
 *              (sum_q w_q |det J_e| K_{e,q}) G_a . (sum_b lambda_{e,b} G_b)
 * where G_b = J_e^{-T} grad_ref phi_b. The per-element part of du equals the
 * Laplacian element residual of the field lambda_e (the element operator is
 * symmetric); it is written to `scratch` and then summed per vertex through the
 * vertex-to-cell lists of fem_build_node2cell, in a fixed order (bitwise
 * reproducible, no atomics).
 *   lambda     [dim+1][C]            adjoint weights per element dof
 *   dK         [n_q][C]              written
 *   du         [V]                   written
 *   node_ptr   [V+1], node_idx [(dim+1)*C]  from fem_build_node2cell for this conn
 *   scratch    [dim+1][C] value type, caller-owned workspace (contents overwritten)
 * Other arguments as fem_integrate_laplacian.
 * ------------------------------------------------------------------------------- */
fem_status fem_adjoint_laplacian(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                 const int32_t *conn, const void *u, const void *K, int n_q,
                                 const double *qpts, const double *qw, const void *lambda, void *dK,
                                 void *du, const int32_t *node_ptr, const int32_t *node_idx,
                                 void *scratch, fem_precision prec, fem_stream stream);

/* ---------------------------------------------------------------------------------
 * fem_adjoint_laplacian_noalloc -- fem_adjoint_laplacian for callers that cannot
 * allocate device memory. The paper has no counterpart; this is a library convenience.
 *
 * Who needs it: callers that have no workspace buffer to pass as `scratch` and cannot
 * get one -- code handed only the input and output pointers (a plugin or callback in
 * a host framework that owns all device memory), or a loop that must not call
 * cudaMalloc because of the device-wide synchronisation it implies.
 *
 * The workspace comes from a fixed array of FEM_NOALLOC_SCRATCH_BYTES in the library's
 * own device memory (a file-scope __device__ object, held by every GPU that loads the
 * library until the process exits). Nothing is allocated: no cudaMalloc, no cudaFree.
 *   - Limit: (dim+1) * n_cells * sizeof(value) must not exceed FEM_NOALLOC_SCRATCH_BYTES
 *     (16 MiB: up to 1,048,576 tets or 1,398,101 triangles in the float32 forms,
 *     524,288 tets or 699,050 triangles in float64 and FEM_FP64_DF); larger calls
 *     return FEM_ERR_SHAPE with a message and launch nothing.
 *   - Set-up: the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call before
 *     any stream capture. The address is kept for the life of the process, so resetting
 *     the device (cudaDeviceReset) after the first call is not supported.
 *   - Sharing: every call on a device uses the same array, which keeps the last call's
 *     contents. Each call writes every entry it reads before reading it, so nothing
 *     needs clearing; but calls that overlap on the GPU (different streams, or host
 *     threads) race on the array and must be serialised by the caller.
 *   - Validity: dK and du are valid only if the next fem_device_error() returns FEM_OK.
 *     A bounded wait that gave up (FEM_ERR_TIMEOUT) leaves a tile of the array unwritten,
 *     and du then includes the previous call's values for it.
 * Arguments, layouts and results are those of fem_adjoint_laplacian without `scratch`.
 * ------------------------------------------------------------------------------- */
#define FEM_NOALLOC_SCRATCH_BYTES (16u << 20)
fem_status fem_adjoint_laplacian_noalloc(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                                         const int32_t *conn, const void *u, const void *K, int n_q,
                                         const double *qpts, const double *qw, const void *lambda, void *dK,
                                         void *du, const int32_t *node_ptr, const int32_t *node_idx,
                                         fem_precision prec, fem_stream stream);

/* ---------------------------------------------------------------------------------
 * fem_build_node2cell -- vertex-to-(cell, local vertex) lists: the transpose of conn,
 * i.e. the assembly operator E_e of Eq. 2 stored as lists. Built on the device,
 * deterministically:
 *   node_ptr [V+1]            node_ptr[n] .. node_ptr[n+1] delimit vertex n's entries
 *   node_idx [(dim+1)*C]      entries e*(dim+1) + a (cell e, local vertex a), sorted
 *                             ascending within each vertex, i.e. in cell order
 *   work     int32 workspace of fem_node2cell_work_size(V) entries
 * All three are caller-owned device arrays. conn must be valid (see fem_check_mesh).
 * ------------------------------------------------------------------------------- */
int64_t fem_node2cell_work_size(int64_t n_verts);
fem_status fem_build_node2cell(int dim, int64_t n_cells, int64_t n_verts, const int32_t *conn,
                               int32_t *node_ptr, int32_t *node_idx, int32_t *work, fem_stream stream);

/* ---------------------------------------------------------------------------------
 * fem_gather_nodes -- the assembly sum E^T of Eq. 2 for element vectors:
 *   out[k][n] = sum over the entries e*(dim+1) + a of vertex n (in list order) of
 *               elem[(a*n_comp + k)*C + e]
 * elem is [(dim+1)*n_comp][C] (the layout of the integrate outputs: n_comp = 1 for the
 * Laplacian, dim for elasticity), out is [n_comp][V]; both of the value type of prec
 * (float64 for FEM_FP64 and FEM_FP64_DF, float32 otherwise). Fixed summation order, no
 * atomics, so repeated calls give bitwise the same out; float64 sums are plain, float32
 * sums compensated (TwoSum). node_ptr / node_idx from fem_build_node2cell for the conn
 * that produced elem.
 * ------------------------------------------------------------------------------- */
fem_status fem_gather_nodes(int dim, int n_comp, int64_t n_cells, int64_t n_verts, const void *elem,
                            const int32_t *node_ptr, const int32_t *node_idx, void *out,
                            fem_precision prec, fem_stream stream);

/* ---------------------------------------------------------------------------------
 * Device-memory arena for the serving loop (not in the paper). A host-side first-fit
 * sub-allocator of offsets into ONE caller-owned device buffer of `capacity` bytes;
 * it makes no CUDA call and never touches the buffer. Offsets are multiples of
 * `alignment` (a power of two); sizes are rounded up to it. Released ranges merge
 * with free neighbours. Thread-safe.
 *   fem_arena_alloc  FEM_ERR_OOM when no free range holds `bytes`
 *   fem_arena_free   FEM_ERR_ARG when `offset` was not returned by fem_arena_alloc
 * ------------------------------------------------------------------------------- */
typedef struct fem_arena fem_arena;
fem_status fem_arena_create(int64_t capacity, int64_t alignment, fem_arena **out);
void fem_arena_destroy(fem_arena *arena);
fem_status fem_arena_alloc(fem_arena *arena, int64_t bytes, int64_t *offset);
fem_status fem_arena_free(fem_arena *arena, int64_t offset);
int64_t fem_arena_free_bytes(fem_arena *arena);
int64_t fem_arena_largest_free(fem_arena *arena);
int64_t fem_arena_capacity(fem_arena *arena);

/* ---------------------------------------------------------------------------------
 * Serving: the per-request launch of a continuous-batching loop (not in the paper).
 * A request's device arrays live in one block (e.g. an fem_arena range of a caller-owned
 * buffer); offset[] gives each array's byte offset in the block, indexed by the
 * FEM_SERVE_* slots (unused slots are ignored). Its inputs (coords, conn, u, K or
 * lambda and mu, adjoint weights) occupy the leading in_bytes of the block and are
 * uploaded from host_in, a page-locked host block with the same layout.
 *
 * fem_serve_launch -- on `stream`: upload host_in (one copy), run the request's kernels
 *   (kind 0: fem_integrate_laplacian or fem_integrate_elasticity; kind 1, Laplacian only:
 *   fem_build_node2cell then fem_adjoint_laplacian; kind 2: the bounded-wait self-test of
 *   fem_selftest_wait with a 1 ms budget and no arrays -- a request that always fails with
 *   the timeout bit, for tests of the failure path), copy out_bytes[0] from slot
 *   OUT (element vectors, or dK) to host_out[0] and out_bytes[1] from slot DU (du) to
 *   host_out[1], then record `event` (from fem_serve_event_create). With host_status set,
 *   the request's kernels report their device-side errors into that word instead of the
 *   device-wide word of fem_device_error: a 4-byte word of page-locked, device-mapped host
 *   memory (cudaHostAlloc, pinned tensors; otherwise FEM_ERR_ARG) that the caller sets to
 *   0 before the launch. Once the event has completed it holds the request's error bits:
 *   0 = none, 1 = a bounded wait gave up (outputs incomplete), 2 = invalid mesh (a vertex
 *   id outside [0, n_verts) or a degenerate cell). Returns after enqueueing; errors as the entry
 *   points it calls. Before any copy or launch the descriptor is checked against the
 *   block: every array the request uses (sizes from dim, n_q, n_cells, n_verts and prec)
 *   must lie inside [0, block_bytes), in_bytes must not exceed block_bytes and
 *   out_bytes[k] must not exceed its source array; otherwise FEM_ERR_ARG and nothing is
 *   enqueued.
 * fem_serve_events_query -- done[i] = 1 if events[i] has completed, else 0.
 * ------------------------------------------------------------------------------- */
enum {
    FEM_SERVE_COORDS = 0, FEM_SERVE_CONN = 1, FEM_SERVE_U = 2,
    FEM_SERVE_K = 3,        /* K, or lambda for elasticity */
    FEM_SERVE_MU = 4, FEM_SERVE_ADJ = 5,
    FEM_SERVE_OUT = 6,      /* element vectors, or dK for the adjoint */
    FEM_SERVE_DU = 7, FEM_SERVE_SCRATCH = 8, FEM_SERVE_NODE_PTR = 9, FEM_SERVE_NODE_IDX = 10,
    FEM_SERVE_WORK = 11,    /* int32 workspace of fem_node2cell_work_size(n_verts) entries */
    FEM_SERVE_SLOTS = 12
};
typedef struct {
    int32_t kind;           /* 0 residual, 1 adjoint, 2 bounded-wait self-test */
    int32_t physics;        /* 0 Laplacian, 1 elasticity */
    int32_t dim, n_q, prec, reserved;
    int64_t n_cells, n_verts;
    const double *qpts, *qw; /* host quadrature tables [n_q][dim], [n_q] */
    const void *host_in;
    int64_t in_bytes;
    void *host_out[2];
    int64_t out_bytes[2];
    int64_t offset[FEM_SERVE_SLOTS];
    int64_t block_bytes;    /* size of the device block the offsets point into */
    void *host_status;      /* device-mapped page-locked uint32 host word for the request's error
                               bits (zeroed by the caller before the launch), or NULL */
} fem_serve_request;
int64_t fem_serve_request_bytes(void); /* sizeof(fem_serve_request), for bindings to check their layout */
fem_status fem_serve_event_create(void **event);
void fem_serve_event_destroy(void *event);
fem_status fem_serve_events_query(void *const *events, int n, int *done);
fem_status fem_serve_launch(const fem_serve_request *request, void *block, void *event, fem_stream stream);

/* fem_serve_run -- a whole request stream served in native code, with the scheduling of
 * the serving loop (continuous batching; not in the paper). Request r arrives arrival[r]
 * seconds (0 <= arrival < 1e9) after the call starts and joins a FIFO queue. A queued request
 * is admitted as soon as one of n_slots (1..FEM_SERVE_MAX_SLOTS) slots -- a stream and a
 * completion event, created and destroyed by the call -- is free and a first-fit arena over
 * `pool` (device memory, pool_bytes bytes, aligned to `alignment`: a power of two >= 256)
 * holds footprint[r] bytes rounded up to `alignment`; with backfill != 0 a later request that
 * fits overtakes a head that does not. Admission zeroes *host_status (if set) and launches
 * reqs[r] with fem_serve_launch into its block (block_bytes taken from footprint[r]);
 * completion is observed by polling the events, and the call returns when every request has
 * finished. results[r] (caller-owned, n entries) receives t_arrive, t_admit, t_done in
 * seconds from the start of the loop (-1 where the request did not get that far), status
 * (FEM_SERVE_DONE; FEM_SERVE_REJECTED: its footprint exceeds the arena, on arrival;
 * FEM_SERVE_FAILED: its kernels set device error bits, in `bits`, see fem_serve_launch;
 * FEM_SERVE_REFUSED: fem_serve_launch refused its descriptor, an argument error, and the
 * stream went on). Returns FEM_ERR_ARG for bad arguments (before anything runs) and
 * FEM_ERR_CUDA when the runtime fails (an event query or enqueue error; the requests in
 * flight are waited for before it returns). */
#define FEM_SERVE_MAX_SLOTS 64
enum { FEM_SERVE_DONE = 0, FEM_SERVE_REJECTED = 1, FEM_SERVE_FAILED = 2, FEM_SERVE_REFUSED = 3 };
typedef struct {
    double t_arrive, t_admit, t_done;
    int32_t status;
    uint32_t bits;
} fem_serve_result;
fem_status fem_serve_run(const fem_serve_request *reqs, const int64_t *footprint, const double *arrival, int n,
                         void *pool, int64_t pool_bytes, int64_t alignment, int n_slots, int backfill,
                         fem_serve_result *results);

/* ---------------------------------------------------------------------------------
 * Throughput probes for the roofline (not part of the method): each thread runs
 * `iters` iterations of 8 independent dependent chains of the chosen operation and
 * writes one value to out[thread] (float64 or float32 as the kind's type).
 *   kind 0: float64 FMA   kind 1: float32 FMA   kind 2: float64 -> float32 conversion
 *   kind 3: 32-bit integer add/logic (LOP3 + IADD pairs)
 * n_threads > 0, multiple of 256.
 * ------------------------------------------------------------------------------- */
fem_status fem_probe(int kind, int64_t n_threads, int iters, void *out, fem_stream stream);

/* ---------------------------------------------------------------------------------
 * fem_device_error -- the device-side status of the kernels since the last call: a
 * per-device error word that kernels set bits in. Two conditions: (1) bounded waits (not
 * in the paper): the staged kernels wait on the bulk copies of their inputs with a time
 * budget (0.5 s per wait); a wait that runs out stops that CTA without writing the tile
 * it waited for; (2) the mesh check (the boundary's debug check, always on): a vertex id
 * outside [0, n_verts) (clamped, so nothing is read out of bounds), or a cell with
 * det J = 0, a non-finite det J or a repeated vertex id. fem_device_error synchronises
 * `stream`, reads and clears the word of the current device, and returns
 * FEM_ERR_TIMEOUT if any wait gave up since the last call (outputs of the calls in
 * between are then incomplete), else FEM_ERR_BADMESH if a kernel met an invalid mesh
 * (the outputs of the cells concerned are meaningless; the others are unaffected), else
 * FEM_OK. Requests of the serving launch report into their own words (fem_serve_launch),
 * not into this one.
 * ------------------------------------------------------------------------------- */
fem_status fem_device_error(fem_stream stream);

/* fem_selftest_wait -- launches one CTA that waits, with the bounded wait of the staged
 * kernels and a budget of budget_ns (0 .. 10 s), for a barrier phase that never
 * completes, so that the next fem_device_error() returns FEM_ERR_TIMEOUT. For tests of
 * the timeout path; it faults nothing and leaves the context usable. */
fem_status fem_selftest_wait(int64_t budget_ns, fem_stream stream);

/* fem_selftest_quotient -- the float64 kernels' division num / |det J| on the device, for
 * tests of its accuracy: q_lib[i] = the library's quotient of num[i] by |den[i]| (a float32
 * seed of the reciprocal refined by two float64 Newton-Raphson steps, the IEEE division
 * for |den| outside [2^-1000, 2^1001), zero, subnormal, infinite or NaN), q_ieee[i] =
 * num[i] / fabs(den[i]) with CUDA's IEEE division. All four arrays are [n] float64 device
 * arrays. */
fem_status fem_selftest_quotient(int64_t n, const double *num, const double *den, double *q_lib, double *q_ieee,
                                 fem_stream stream);

/* status text and the thread-local message of the last failing call */
const char *fem_status_string(fem_status st);
const char *fem_last_error(void);
/* library version string */
const char *fem_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FEM_H */
