"""Closed forms used to pin the oracle (test helper, numpy only).

None of this shares a code path with the oracle: the P1 gradients come from
inverting the barycentric matrix M (rows [1, x_b^T]) with LAPACK instead of a
Jacobian adjugate, and integrals of polynomial coefficients come from the exact
simplex moment formulas instead of a quadrature rule:

  int_T 1      = |T|
  int_T x_i    = |T| xbar_i
  int_T x_i x_j = |T| / ((d+1)(d+2)) [ sum_b x_bi x_bj + (sum_b x_bi)(sum_b x_bj) ]

(the last from int_T lambda_a lambda_b = |T| d! (1 + delta_ab) / (d+2)!).
"""

from __future__ import annotations

import math

import numpy as np


def cell_vertices(coords, conn):
    """(C, d+1, d) vertex coordinates per cell."""
    return np.transpose(coords[:, conn], (2, 1, 0))


def p1_gradients(coords, conn):
    """Physical P1 gradients (C, d+1, d) and cell volumes (C,) via M^{-1}."""
    X = cell_vertices(coords, conn)
    C, nb, d = X.shape
    M = np.concatenate([np.ones((C, nb, 1)), X], axis=2)  # rows [1, x_b]
    Minv = np.linalg.inv(M)  # column b holds (a_b, g_b) of phi_b = a_b + g_b . x
    grads = np.transpose(Minv[:, 1:, :], (0, 2, 1))  # (C, b, d)
    vol = np.abs(np.linalg.det(M)) / math.factorial(d)
    return grads, vol


def quadratic_integral(coords, conn, k0, g, H):
    """int_T (k0 + g.x + x^T H x) dx per cell, exactly."""
    X = cell_vertices(coords, conn)
    C, nb, d = X.shape
    _, vol = p1_gradients(coords, conn)
    xbar = X.mean(axis=1)
    S = X.sum(axis=1)  # (C, d)
    second = (np.einsum("cbi,cbj->cij", X, X) + np.einsum("ci,cj->cij", S, S)) / ((d + 1) * (d + 2))
    return vol * (k0 + xbar @ g + np.einsum("cij,ij->c", second, H))


def quadratic_at(xq, k0, g, H):
    """Evaluate k0 + g.x + x^T H x at points xq of shape (..., d, C) -> (..., C)."""
    lin = np.einsum("i,...ic->...c", g, xq)
    quad = np.einsum("...ic,ij,...jc->...c", xq, H, xq)
    return k0 + lin + quad


def laplacian_exact(coords, conn, u, intK):
    """r_b = (int_T K) grad phi_b . grad u for P1 (constant gradients), shape (d+1, C)."""
    G, _ = p1_gradients(coords, conn)
    ub = u[conn].T  # (C, b)
    gradu = np.einsum("cb,cbi->ci", ub, G)
    return (intK[:, None] * np.einsum("cbi,ci->cb", G, gradu)).T


def elasticity_exact(coords, conn, u, intlam, intmu):
    """r_{b,k} = sum_i G_{b,i} (tr eps delta_ki int lambda + 2 eps_ki int mu), shape ((d+1) d, C)."""
    G, _ = p1_gradients(coords, conn)
    d = coords.shape[0]
    ub = np.transpose(u[:, conn], (2, 1, 0))  # (C, b, k)
    gradu = np.einsum("cbk,cbi->cki", ub, G)
    eps = 0.5 * (gradu + np.transpose(gradu, (0, 2, 1)))
    tr = np.trace(eps, axis1=1, axis2=2)
    sigma = intlam[:, None, None] * tr[:, None, None] * np.eye(d)[None] + 2.0 * intmu[:, None, None] * eps
    r = np.einsum("cki,cbi->cbk", sigma, G)  # (C, b, k)
    return r.reshape(r.shape[0], -1).T


def triangle_stiffness(x):
    """Textbook P1 stiffness of one triangle with vertices x (3, 2):
    A_ij = (b_i b_j + c_i c_j) / (4 |T|), b_i = y_j - y_k, c_i = x_k - x_j (i, j, k cyclic)."""
    b = np.array([x[(i + 1) % 3, 1] - x[(i + 2) % 3, 1] for i in range(3)])
    c = np.array([x[(i + 2) % 3, 0] - x[(i + 1) % 3, 0] for i in range(3)])
    area = 0.5 * abs((x[1, 0] - x[0, 0]) * (x[2, 1] - x[0, 1]) - (x[2, 0] - x[0, 0]) * (x[1, 1] - x[0, 1]))
    return (np.outer(b, b) + np.outer(c, c)) / (4.0 * area)


def assemble(conn, elem, n_verts, n_comp=1):
    """E^T: sum element vectors (rows b*n_comp + k) into a nodal vector (n_comp, V)."""
    out = np.zeros((n_comp, n_verts))
    nb = conn.shape[0]
    for b in range(nb):
        for k in range(n_comp):
            np.add.at(out[k], conn[b], elem[b * n_comp + k])
    return out


def min_det(coords, conn):
    """Smallest signed det of the edge matrix over all cells (numpy det, independent)."""
    X = cell_vertices(coords, conn)
    E = X[:, 1:, :] - X[:, :1, :]
    return float(np.linalg.det(E).min())
