/*
 * fem_oracle.c -- plain CPU FP64 oracle for P1 quadrature element integration.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the CUDA
 * library is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table or
 * helper with the CUDA library: it receives the same raw arrays and computes the
 * element integrals the slow, obvious way.
 *
 * What it computes (Knepley, Rupp, Terrel, "Finite Element Integration with
 * Quadrature on the GPU"):
 *
 *   The bracket of Eq. 2 for one cell e, with f0 = 0:
 *       r_e = sum_k D_k^T W f1^k(u^q, grad u^q)
 *   i.e. for every basis function b of the cell
 *       r_{e,b} = sum_q w_q |det J| (J^{-T} grad_ref phi_b(xi_q)) . f1(q)
 *   with the pointwise functions of Sec. 2 / Sec. 6:
 *       Laplacian   f1 = K(x_q) grad u                       (variable coefficient)
 *       elasticity  f1 = lambda tr(eps) I + 2 mu eps,  eps = (grad u + grad u^T)/2
 *   (with lambda = 0, mu = 1/2 this is the paper's symmetric-gradient listing).
 *
 *   Per cell the steps follow the order of Sec. 3 and the Appendix: load the
 *   geometry and the basis coefficients of the cell, evaluate grad u at each
 *   quadrature point with the tabulated reference derivatives, apply the pointwise
 *   function and scale it by the weight and the determinant (quadrature phase,
 *   Sec. 3.1), then contract with the test-function gradients, summing over the
 *   quadrature points in index order (basis phase, Sec. 3.2).
 *
 *   The paper loads a precomputed inverse Jacobian and determinant; here they are
 *   computed from the vertex coordinates: J = [x_1 - x_0 | ... | x_d - x_0]
 *   (J_ij = dx_i/dxi_j), det J by cofactor expansion along the first row, and
 *   J^{-1} = adj(J) / det J.  Readings of points the paper leaves open: the
 *   determinant enters as |det J|, and physical gradients are J^{-T} grad_ref phi.
 *
 *   Adjoint (not in the paper): for the scalar J(u, K) = sum_e sum_b lambda_{e,b} r_{e,b},
 *       dJ/dK_{e,q} = w_q |det J| (sum_b lambda_{e,b} G_b(q)) . grad u(q)
 *       dJ/du_n     = sum over (e, a) with conn(e, a) = n of sum_b lambda_{e,b} A_e[b][a]
 *   where G_b(q) = J^{-T} grad_ref phi_b(xi_q) and A_e[b][a] = sum_q w_q |det J| K_{e,q}
 *   G_b(q).G_a(q) is the element stiffness matrix (dr_{e,b}/du_{e,a}; r is linear in u).
 *
 * Array layout (structure of arrays, the fastest index last in the name):
 *   coords [dim][n_verts], conn [dim+1][n_cells] (int32 vertex ids),
 *   u      [n_verts] (Laplacian) or [dim][n_verts] (elasticity),
 *   K, lam, mu [n_q][n_cells], qpts [n_q][dim], qw [n_q],
 *   out    [(dim+1)*n_comp][n_cells] with row b*n_comp + k,
 *   lambda [dim+1][n_cells], dK [n_q][n_cells], du [n_verts].
 *
 * Return value: 0 on success, -1 bad argument, -5 bad mesh (vertex id out of range
 * or a cell with det J = 0).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_MAX_Q 64
#define ORA_OK 0
#define ORA_ERR_ARG (-1)
#define ORA_ERR_BADMESH (-5)

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Thread count of the loops over cells (timing only; the results do not depend on it:
 * every cell is computed by one thread, in the same order of operations). */
void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* P1 basis on the reference simplex, evaluated at the quadrature points:
 * phi_0 = 1 - sum_k xi_k, phi_b = xi_{b-1}; their reference gradients are
 * d phi_0 / d xi_k = -1 and d phi_b / d xi_k = [k == b-1].  The tables are built per
 * point, the way the paper tabulates Basis_0[q,b] and BasisDerivatives_0[q,b]. */
static void tabulate_p1(int dim, int n_q, const double *qpts, double phi[][4], double dphi[][4][3]) {
    for (int q = 0; q < n_q; ++q) {
        double s = 0.0;
        for (int k = 0; k < dim; ++k) s += qpts[q * dim + k];
        phi[q][0] = 1.0 - s;
        for (int k = 0; k < dim; ++k) dphi[q][0][k] = -1.0;
        for (int b = 1; b <= dim; ++b) {
            phi[q][b] = qpts[q * dim + (b - 1)];
            for (int k = 0; k < dim; ++k) dphi[q][b][k] = (k == b - 1) ? 1.0 : 0.0;
        }
    }
}

static int check_args(int dim, int64_t n_cells, int64_t n_verts, int n_q) {
    if (dim != 2 && dim != 3) return ORA_ERR_ARG;
    if (n_cells < 0 || n_verts < 0) return ORA_ERR_ARG;
    if (n_q < 1 || n_q > ORA_MAX_Q) return ORA_ERR_ARG;
    return ORA_OK;
}

static int check_conn(int dim, int64_t n_cells, int64_t n_verts, const int32_t *conn) {
    for (int64_t i = 0; i < (int64_t)(dim + 1) * n_cells; ++i)
        if (conn[i] < 0 || (int64_t)conn[i] >= n_verts) return ORA_ERR_BADMESH;
    return ORA_OK;
}

/* Geometry of cell c: vertex coordinates x[b][i], the Jacobian J[i][j] = x_{j+1,i} - x_{0,i},
 * its determinant (cofactor expansion along row 0) and its inverse adj(J)/det J. */
static double cell_geometry(int dim, int64_t c, int64_t n_cells, int64_t n_verts, const double *coords,
                            const int32_t *conn, double J[3][3], double invJ[3][3]) {
    double x[4][3];
    for (int b = 0; b <= dim; ++b) {
        int64_t v = conn[(int64_t)b * n_cells + c];
        for (int i = 0; i < dim; ++i) x[b][i] = coords[(int64_t)i * n_verts + v];
    }
    for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) J[i][j] = x[j + 1][i] - x[0][i];
    double det;
    if (dim == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        if (det == 0.0) return 0.0;
        /* adj(J) = [[J11, -J01], [-J10, J00]] */
        invJ[0][0] = J[1][1] / det;
        invJ[0][1] = -J[0][1] / det;
        invJ[1][0] = -J[1][0] / det;
        invJ[1][1] = J[0][0] / det;
    } else {
        double cof[3][3]; /* cof[i][j] = (-1)^(i+j) * minor(i, j) */
        cof[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        cof[0][1] = -(J[1][0] * J[2][2] - J[1][2] * J[2][0]);
        cof[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        cof[1][0] = -(J[0][1] * J[2][2] - J[0][2] * J[2][1]);
        cof[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
        cof[1][2] = -(J[0][0] * J[2][1] - J[0][1] * J[2][0]);
        cof[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
        cof[2][1] = -(J[0][0] * J[1][2] - J[0][2] * J[1][0]);
        cof[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        det = J[0][0] * cof[0][0] + J[0][1] * cof[0][1] + J[0][2] * cof[0][2];
        if (det == 0.0) return 0.0;
        /* adj(J) = cof^T */
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) invJ[i][j] = cof[j][i] / det;
    }
    return det;
}

/* Physical gradient of basis b at point q: G_i = sum_k invJ[k][i] dphi[q][b][k]  (J^{-T} grad_ref). */
static void phys_grad(int dim, const double invJ[3][3], const double dref[3], double G[3]) {
    for (int i = 0; i < dim; ++i) {
        double s = 0.0;
        for (int k = 0; k < dim; ++k) s += invJ[k][i] * dref[k];
        G[i] = s;
    }
}

int oracle_laplacian(int dim, int64_t n_cells, int64_t n_verts, const double *coords, const int32_t *conn,
                     const double *u, const double *K, int n_q, const double *qpts, const double *qw,
                     double *out) {
    int st = check_args(dim, n_cells, n_verts, n_q);
    if (st) return st;
    if (n_cells == 0) return ORA_OK;
    if (!coords || !conn || !u || !K || !qpts || !qw || !out) return ORA_ERR_ARG;
    if ((st = check_conn(dim, n_cells, n_verts, conn))) return st;
    const int nb = dim + 1;
    double phi[ORA_MAX_Q][4], dphi[ORA_MAX_Q][4][3];
    tabulate_p1(dim, n_q, qpts, phi, dphi);
    int bad = 0;
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n_cells; ++c) {
        double J[3][3], invJ[3][3];
        double detJ = cell_geometry(dim, c, n_cells, n_verts, coords, conn, J, invJ);
        if (detJ == 0.0) {
#pragma omp atomic write
            bad = 1;
            continue;
        }
        double ub[4];
        for (int b = 0; b < nb; ++b) ub[b] = u[conn[(int64_t)b * n_cells + c]];
        /* quadrature phase: f1 at every point, scaled by w_q |det J| */
        double f1[ORA_MAX_Q][3];
        for (int q = 0; q < n_q; ++q) {
            double gradU[3] = {0.0, 0.0, 0.0};
            for (int b = 0; b < nb; ++b) {
                double G[3];
                phys_grad(dim, invJ, dphi[q][b], G);
                for (int i = 0; i < dim; ++i) gradU[i] += ub[b] * G[i];
            }
            double kq = K[(int64_t)q * n_cells + c];
            for (int i = 0; i < dim; ++i) f1[q][i] = kq * gradU[i] * qw[q] * fabs(detJ);
        }
        /* basis phase: e_b = sum_q G_b(q) . f1(q) */
        for (int b = 0; b < nb; ++b) {
            double e = 0.0;
            for (int q = 0; q < n_q; ++q) {
                double G[3];
                phys_grad(dim, invJ, dphi[q][b], G);
                for (int i = 0; i < dim; ++i) e += G[i] * f1[q][i];
            }
            out[(int64_t)b * n_cells + c] = e;
        }
    }
    return bad ? ORA_ERR_BADMESH : ORA_OK;
}

int oracle_elasticity(int dim, int64_t n_cells, int64_t n_verts, const double *coords, const int32_t *conn,
                      const double *u, const double *lam, const double *mu, int n_q, const double *qpts,
                      const double *qw, double *out) {
    int st = check_args(dim, n_cells, n_verts, n_q);
    if (st) return st;
    if (n_cells == 0) return ORA_OK;
    if (!coords || !conn || !u || !lam || !mu || !qpts || !qw || !out) return ORA_ERR_ARG;
    if ((st = check_conn(dim, n_cells, n_verts, conn))) return st;
    const int nb = dim + 1;
    double phi[ORA_MAX_Q][4], dphi[ORA_MAX_Q][4][3];
    tabulate_p1(dim, n_q, qpts, phi, dphi);
    int bad = 0;
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n_cells; ++c) {
        double J[3][3], invJ[3][3];
        double detJ = cell_geometry(dim, c, n_cells, n_verts, coords, conn, J, invJ);
        if (detJ == 0.0) {
#pragma omp atomic write
            bad = 1;
            continue;
        }
        /* basis coefficients u_{b,k}: component k of the displacement at vertex b */
        double ub[4][3];
        for (int b = 0; b < nb; ++b) {
            int64_t v = conn[(int64_t)b * n_cells + c];
            for (int k = 0; k < dim; ++k) ub[b][k] = u[(int64_t)k * n_verts + v];
        }
        double f1[ORA_MAX_Q][3][3];
        for (int q = 0; q < n_q; ++q) {
            double gradU[3][3] = {{0}}; /* gradU[k][i] = d u_k / d x_i */
            for (int b = 0; b < nb; ++b) {
                double G[3];
                phys_grad(dim, invJ, dphi[q][b], G);
                for (int k = 0; k < dim; ++k)
                    for (int i = 0; i < dim; ++i) gradU[k][i] += ub[b][k] * G[i];
            }
            double eps[3][3], tr = 0.0;
            for (int k = 0; k < dim; ++k)
                for (int i = 0; i < dim; ++i) eps[k][i] = 0.5 * (gradU[k][i] + gradU[i][k]);
            for (int k = 0; k < dim; ++k) tr += eps[k][k];
            double lq = lam[(int64_t)q * n_cells + c], mq = mu[(int64_t)q * n_cells + c];
            for (int k = 0; k < dim; ++k)
                for (int i = 0; i < dim; ++i) {
                    double sigma = 2.0 * mq * eps[k][i] + (k == i ? lq * tr : 0.0);
                    f1[q][k][i] = sigma * qw[q] * fabs(detJ);
                }
        }
        for (int b = 0; b < nb; ++b) {
            for (int k = 0; k < dim; ++k) {
                double e = 0.0;
                for (int q = 0; q < n_q; ++q) {
                    double G[3];
                    phys_grad(dim, invJ, dphi[q][b], G);
                    for (int i = 0; i < dim; ++i) e += G[i] * f1[q][k][i];
                }
                out[(int64_t)(b * dim + k) * n_cells + c] = e;
            }
        }
    }
    return bad ? ORA_ERR_BADMESH : ORA_OK;
}

int oracle_adjoint_laplacian(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                             const int32_t *conn, const double *u, const double *K, int n_q,
                             const double *qpts, const double *qw, const double *lambda, double *dK,
                             double *du) {
    int st = check_args(dim, n_cells, n_verts, n_q);
    if (st) return st;
    if (!du && n_verts > 0) return ORA_ERR_ARG;
    for (int64_t v = 0; v < n_verts; ++v) du[v] = 0.0;
    if (n_cells == 0) return ORA_OK;
    if (!coords || !conn || !u || !K || !qpts || !qw || !lambda || !dK) return ORA_ERR_ARG;
    if ((st = check_conn(dim, n_cells, n_verts, conn))) return st;
    const int nb = dim + 1;
    double phi[ORA_MAX_Q][4], dphi[ORA_MAX_Q][4][3];
    tabulate_p1(dim, n_q, qpts, phi, dphi);
    double *du_e = (double *)malloc(sizeof(double) * (size_t)nb * (size_t)n_cells);
    if (!du_e) return ORA_ERR_ARG;
    int bad = 0;
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n_cells; ++c) {
        double J[3][3], invJ[3][3];
        double detJ = cell_geometry(dim, c, n_cells, n_verts, coords, conn, J, invJ);
        if (detJ == 0.0) {
#pragma omp atomic write
            bad = 1;
            continue;
        }
        double ub[4], lb[4];
        for (int b = 0; b < nb; ++b) {
            ub[b] = u[conn[(int64_t)b * n_cells + c]];
            lb[b] = lambda[(int64_t)b * n_cells + c];
        }
        double A[4][4] = {{0}};
        for (int q = 0; q < n_q; ++q) {
            double G[4][3];
            for (int b = 0; b < nb; ++b) phys_grad(dim, invJ, dphi[q][b], G[b]);
            double gradU[3] = {0, 0, 0}, L[3] = {0, 0, 0};
            for (int b = 0; b < nb; ++b)
                for (int i = 0; i < dim; ++i) {
                    gradU[i] += ub[b] * G[b][i];
                    L[i] += lb[b] * G[b][i];
                }
            double s = 0.0;
            for (int i = 0; i < dim; ++i) s += L[i] * gradU[i];
            dK[(int64_t)q * n_cells + c] = qw[q] * fabs(detJ) * s;
            double kq = K[(int64_t)q * n_cells + c];
            for (int b = 0; b < nb; ++b)
                for (int a = 0; a < nb; ++a) {
                    double g = 0.0;
                    for (int i = 0; i < dim; ++i) g += G[b][i] * G[a][i];
                    A[b][a] += qw[q] * fabs(detJ) * kq * g;
                }
        }
        for (int a = 0; a < nb; ++a) {
            double s = 0.0;
            for (int b = 0; b < nb; ++b) s += lb[b] * A[b][a];
            du_e[(int64_t)a * n_cells + c] = s;
        }
    }
    if (!bad) {
        /* nodal sum, one plain loop over cells in order */
        for (int64_t c = 0; c < n_cells; ++c)
            for (int a = 0; a < nb; ++a) du[conn[(int64_t)a * n_cells + c]] += du_e[(int64_t)a * n_cells + c];
    }
    free(du_e);
    return bad ? ORA_ERR_BADMESH : ORA_OK;
}

/* Reaction-diffusion with an auxiliary coefficient field: the full bracket of Eq. 2,
 *     r_{e,b} = sum_q w_q |det J| [ phi_b(xi_q) f0(q) + G_b(q) . f1(q) ],
 * with the pointwise functions of Eq. 8 taking the auxiliary field a and its gradient:
 *     f1(u, grad u, a) = a grad u,      f0(u, grad u, a, grad a) = c u + g grad a . grad u,
 * evaluated at each quadrature point from the tabulated basis:
 *     u(q) = sum_b phi_b(xi_q) u_b,  grad u(q) = sum_b u_b G_b(q),
 *     a(q) = sum_b phi_b(xi_q) a_b,  grad a(q) = sum_b a_b G_b(q)
 *                                    (a_space = 1: a in P1, nodal values a[V])
 *     a(q) = a_e,  grad a(q) = 0     (a_space = 0: a in P0, one value per cell a[C])
 * c [n_q][C] is the reaction coefficient per quadrature point (c = NULL: no reaction term);
 * g (`drift`) scales the first-order term along grad a (g = 0: none). */
int oracle_reaction_diffusion(int dim, int64_t n_cells, int64_t n_verts, const double *coords,
                              const int32_t *conn, const double *u, const double *a, int a_space,
                              const double *c, double drift, int n_q, const double *qpts, const double *qw,
                              double *out) {
    int st = check_args(dim, n_cells, n_verts, n_q);
    if (st) return st;
    if (a_space != 0 && a_space != 1) return ORA_ERR_ARG;
    if (n_cells == 0) return ORA_OK;
    if (!coords || !conn || !u || !a || !qpts || !qw || !out) return ORA_ERR_ARG;
    if ((st = check_conn(dim, n_cells, n_verts, conn))) return st;
    const int nb = dim + 1;
    double phi[ORA_MAX_Q][4], dphi[ORA_MAX_Q][4][3];
    tabulate_p1(dim, n_q, qpts, phi, dphi);
    int bad = 0;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n_cells; ++e) {
        double J[3][3], invJ[3][3];
        double detJ = cell_geometry(dim, e, n_cells, n_verts, coords, conn, J, invJ);
        if (detJ == 0.0) {
#pragma omp atomic write
            bad = 1;
            continue;
        }
        double ub[4], ab[4];
        for (int b = 0; b < nb; ++b) {
            int64_t v = conn[(int64_t)b * n_cells + e];
            ub[b] = u[v];
            ab[b] = a_space == 1 ? a[v] : a[e];
        }
        /* quadrature phase: f0 and f1 at every point, scaled by w_q |det J| */
        double f0[ORA_MAX_Q], f1[ORA_MAX_Q][3];
        for (int q = 0; q < n_q; ++q) {
            double uq = 0.0, aq = 0.0, gradU[3] = {0.0, 0.0, 0.0}, gradA[3] = {0.0, 0.0, 0.0};
            for (int b = 0; b < nb; ++b) {
                double G[3];
                phys_grad(dim, invJ, dphi[q][b], G);
                uq += phi[q][b] * ub[b];
                aq += phi[q][b] * ab[b];
                for (int i = 0; i < dim; ++i) {
                    gradU[i] += ub[b] * G[i];
                    gradA[i] += ab[b] * G[i];
                }
            }
            if (a_space == 0) {
                aq = ab[0];
                for (int i = 0; i < dim; ++i) gradA[i] = 0.0;
            }
            double scale = qw[q] * fabs(detJ);
            double f0q = c ? c[(int64_t)q * n_cells + e] * uq : 0.0;
            for (int i = 0; i < dim; ++i) f0q += drift * gradA[i] * gradU[i];
            f0[q] = f0q * scale;
            for (int i = 0; i < dim; ++i) f1[q][i] = aq * gradU[i] * scale;
        }
        /* basis phase: e_b = sum_q phi_b(q) f0(q) + G_b(q) . f1(q) */
        for (int b = 0; b < nb; ++b) {
            double r = 0.0;
            for (int q = 0; q < n_q; ++q) {
                double G[3];
                phys_grad(dim, invJ, dphi[q][b], G);
                r += phi[q][b] * f0[q];
                for (int i = 0; i < dim; ++i) r += G[i] * f1[q][i];
            }
            out[(int64_t)b * n_cells + e] = r;
        }
    }
    return bad ? ORA_ERR_BADMESH : ORA_OK;
}

/* Pointwise physics of the caller's choosing: the general bracket of Eq. 2 for a field of
 * n_comp components,
 *     r_{e,b,k} = sum_q w_q |det J| [ phi_b(xi_q) f0_k(q) + sum_i G_{b,i}(q) f1_{k,i}(q) ],
 * with the pointwise functions evaluated at every quadrature point from
 *     u_k(q) = sum_b phi_b(xi_q) u_{b,k},   grad u_{k,i}(q) = sum_b u_{b,k} G_{b,i}(q),
 *     x_i(q) = sum_b phi_b(xi_q) x_{b,i},   a_j(q) = coef[(j*n_q + q)*n_cells + e].
 * The CUDA library takes f0 and f1 as source strings compiled at run time (Sec. 5); the
 * oracle has a fixed set of them, chosen by `physics` (params p[0..3]):
 *   0  f1 = a_0 grad u                                  (the variable-coefficient Laplacian)
 *   1  f1 = kappa(u, x) grad u,  kappa = (p0 + p1 u + p2 u^2)(1 + p3 s(x)),
 *      s(x) = x_0 + 2 x_1 (+ 3 x_2)                     (Sec. 2's nonlinear kappa(u, x) grad u)
 *   2  f1 = a_0 tr(eps) I + 2 a_1 eps, eps = (grad u + grad u^T)/2   (Lame; n_comp = dim)
 *   3  f0 = a_0 u + p0,  f1 = a_1 grad u                (reaction, source and diffusion)
 * u is [n_comp][n_verts], out [(dim+1)*n_comp][n_cells] with row b*n_comp + k. */
static void pointwise_f(int physics, const double *p, int dim, int n_comp, const double *uq, double gu[3][3],
                        const double *xq, const double *aq, double f0[3], double f1[3][3]) {
    for (int k = 0; k < n_comp; ++k) {
        f0[k] = 0.0;
        for (int i = 0; i < dim; ++i) f1[k][i] = 0.0;
    }
    if (physics == 0) {
        for (int i = 0; i < dim; ++i) f1[0][i] = aq[0] * gu[0][i];
    } else if (physics == 1) {
        double sx = 0.0;
        for (int i = 0; i < dim; ++i) sx += (i + 1) * xq[i];
        const double kappa = (p[0] + p[1] * uq[0] + p[2] * uq[0] * uq[0]) * (1.0 + p[3] * sx);
        for (int i = 0; i < dim; ++i) f1[0][i] = kappa * gu[0][i];
    } else if (physics == 2) {
        double eps[3][3], tr = 0.0;
        for (int k = 0; k < dim; ++k)
            for (int i = 0; i < dim; ++i) eps[k][i] = 0.5 * (gu[k][i] + gu[i][k]);
        for (int k = 0; k < dim; ++k) tr += eps[k][k];
        for (int k = 0; k < dim; ++k)
            for (int i = 0; i < dim; ++i) f1[k][i] = 2.0 * aq[1] * eps[k][i] + (k == i ? aq[0] * tr : 0.0);
    } else {
        f0[0] = aq[0] * uq[0] + p[0];
        for (int i = 0; i < dim; ++i) f1[0][i] = aq[1] * gu[0][i];
    }
}

int oracle_pointwise(int physics, const double *params, int dim, int n_comp, int n_coef, int64_t n_cells,
                     int64_t n_verts, const double *coords, const int32_t *conn, const double *u,
                     const double *coef, int n_q, const double *qpts, const double *qw, double *out) {
    int st = check_args(dim, n_cells, n_verts, n_q);
    if (st) return st;
    if (physics < 0 || physics > 3 || n_comp < 1 || n_comp > 3 || n_coef < 0) return ORA_ERR_ARG;
    if ((physics == 2) != (n_comp == dim && n_comp > 1)) return ORA_ERR_ARG;
    const int need_coef = physics == 1 ? 0 : (physics == 0 ? 1 : 2);
    if (n_coef < need_coef) return ORA_ERR_ARG;
    if (n_cells == 0) return ORA_OK;
    if (!coords || !conn || !u || !qpts || !qw || !out || !params || (n_coef > 0 && !coef)) return ORA_ERR_ARG;
    if ((st = check_conn(dim, n_cells, n_verts, conn))) return st;
    const int nb = dim + 1;
    double phi[ORA_MAX_Q][4], dphi[ORA_MAX_Q][4][3];
    tabulate_p1(dim, n_q, qpts, phi, dphi);
    int bad = 0;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n_cells; ++e) {
        double J[3][3], invJ[3][3];
        double detJ = cell_geometry(dim, e, n_cells, n_verts, coords, conn, J, invJ);
        if (detJ == 0.0) {
#pragma omp atomic write
            bad = 1;
            continue;
        }
        double ub[4][3], xb[4][3];
        for (int b = 0; b < nb; ++b) {
            int64_t v = conn[(int64_t)b * n_cells + e];
            for (int k = 0; k < n_comp; ++k) ub[b][k] = u[(int64_t)k * n_verts + v];
            for (int i = 0; i < dim; ++i) xb[b][i] = coords[(int64_t)i * n_verts + v];
        }
        /* quadrature phase: f0 and f1 at every point, scaled by w_q |det J| */
        double f0[ORA_MAX_Q][3], f1[ORA_MAX_Q][3][3];
        for (int q = 0; q < n_q; ++q) {
            double uq[3] = {0, 0, 0}, xq[3] = {0, 0, 0}, gu[3][3] = {{0}}, aq[8] = {0};
            for (int b = 0; b < nb; ++b) {
                double G[3];
                phys_grad(dim, invJ, dphi[q][b], G);
                for (int k = 0; k < n_comp; ++k) {
                    uq[k] += phi[q][b] * ub[b][k];
                    for (int i = 0; i < dim; ++i) gu[k][i] += ub[b][k] * G[i];
                }
                for (int i = 0; i < dim; ++i) xq[i] += phi[q][b] * xb[b][i];
            }
            for (int j = 0; j < n_coef && j < 8; ++j) aq[j] = coef[((int64_t)j * n_q + q) * n_cells + e];
            double g0[3], g1[3][3];
            pointwise_f(physics, params, dim, n_comp, uq, gu, xq, aq, g0, g1);
            const double scale = qw[q] * fabs(detJ);
            for (int k = 0; k < n_comp; ++k) {
                f0[q][k] = g0[k] * scale;
                for (int i = 0; i < dim; ++i) f1[q][k][i] = g1[k][i] * scale;
            }
        }
        /* basis phase: r_{b,k} = sum_q phi_b(q) f0_k(q) + G_b(q) . f1_k(q) */
        for (int b = 0; b < nb; ++b)
            for (int k = 0; k < n_comp; ++k) {
                double r = 0.0;
                for (int q = 0; q < n_q; ++q) {
                    double G[3];
                    phys_grad(dim, invJ, dphi[q][b], G);
                    r += phi[q][b] * f0[q][k];
                    for (int i = 0; i < dim; ++i) r += G[i] * f1[q][k][i];
                }
                out[(int64_t)(b * n_comp + k) * n_cells + e] = r;
            }
    }
    return bad ? ORA_ERR_BADMESH : ORA_OK;
}
