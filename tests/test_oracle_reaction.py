"""Pins of the oracle's reaction-diffusion routine (Eq. 2 with both terms; Eq. 8: the
pointwise functions take an auxiliary field a in P1 or P0 and its gradient):
f1 = a grad u, f0 = c u + g grad a . grad u.

Each check compares against something other than the routine itself: the already
pinned Laplacian routine (a in P0, no reaction), the exact P1 stiffness with the exact
mean of a linear a, the closed-form P1 mass matrix, the exact integral of f0 over the
cell, symmetry of the assembled operator, and for the grad a term the exact integral
g (p.s) |T|/(d+1) for linear fields with gradients p and s, its symmetry in u and a, and
its absence for a P0 coefficient.
"""

import math

import numpy as np
import pytest

import workloads

import exact


def _random_simplices(dim, n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, dim + 1, dim))
    coords = X.reshape(-1, dim).T.copy()
    conn = np.arange(n * (dim + 1), dtype=np.int32).reshape(n, dim + 1).T.copy()
    return coords, conn


@pytest.mark.parametrize("dim", [2, 3])
def test_p0_coefficient_without_reaction_is_the_laplacian(ora, dim):
    coords, conn = _random_simplices(dim, 40, 3 + dim)
    rule = workloads.rule_for_dim(dim)
    rng = np.random.default_rng(dim)
    u = rng.uniform(-1, 1, coords.shape[1])
    a = rng.lognormal(0, 1, conn.shape[1])
    r = ora.reaction_diffusion(coords, conn, u, a, 0, None, rule.points, rule.weights)
    ref = ora.laplacian(coords, conn, u, np.tile(a, (rule.n_q, 1)), rule.points, rule.weights)
    assert np.abs(r - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_linear_p1_coefficient_exact(ora, dim):
    """a linear in x: a grad phi_b . grad u is linear, so the degree-2 rule is exact and
    r_b = |T| a(centroid) G_b . g with G_b the exact P1 gradients."""
    coords, conn = _random_simplices(dim, 50, 11 * dim)
    rule = workloads.rule_for_dim(dim)
    rng = np.random.default_rng(5)
    u = rng.uniform(-1, 1, coords.shape[1])
    alpha, beta = 2.0, rng.normal(size=dim)
    a = alpha + beta @ coords  # nodal values of a linear field
    r = ora.reaction_diffusion(coords, conn, u, a, 1, None, rule.points, rule.weights)
    G, vol = exact.p1_gradients(coords, conn)
    xbar = exact.cell_vertices(coords, conn).mean(axis=1)  # (C, d)
    abar = alpha + xbar @ beta
    g = np.einsum("cb,cbi->ci", u[conn].T, G)
    ref = (vol * abar)[None, :] * np.einsum("cbi,ci->bc", G, g)
    assert np.abs(r - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_mass_term_closed_form(ora, dim):
    """a = 0, c = gamma per cell: r = gamma M u with M_ab = |T| (1 + delta_ab) / ((d+1)(d+2))."""
    coords, conn = _random_simplices(dim, 30, 17 + dim)
    rule = workloads.rule_for_dim(dim)
    rng = np.random.default_rng(9)
    C = conn.shape[1]
    u = rng.uniform(-1, 1, coords.shape[1])
    gamma = rng.uniform(0.5, 2.0, C)
    c = np.tile(gamma, (rule.n_q, 1))
    r = ora.reaction_diffusion(coords, conn, u, np.zeros(C), 0, c, rule.points, rule.weights)
    _, vol = exact.p1_gradients(coords, conn)
    nb = dim + 1
    M = (np.ones((nb, nb)) + np.eye(nb)) / ((dim + 1) * (dim + 2))
    ref = (gamma * vol)[None, :] * (M @ u[conn])
    assert np.abs(r - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_element_sums_equal_the_integral_of_f0(ora, dim):
    """sum_b phi_b = 1 and sum_b grad phi_b = 0, so sum_b r_b = int_T c u = c |T| mean(u_b)."""
    coords, conn = _random_simplices(dim, 30, 23 + dim)
    rule = workloads.rule_for_dim(dim)
    rng = np.random.default_rng(2)
    C, V = conn.shape[1], coords.shape[1]
    u, a = rng.uniform(-1, 1, V), rng.lognormal(0, 1, V)
    gamma = rng.uniform(0.5, 2.0, C)
    r = ora.reaction_diffusion(coords, conn, u, a, 1, np.tile(gamma, (rule.n_q, 1)), rule.points, rule.weights)
    _, vol = exact.p1_gradients(coords, conn)
    ref = gamma * vol * u[conn].mean(axis=0)
    assert np.abs(r.sum(axis=0) - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_assembled_operator_symmetric(ora, dim):
    mesh = workloads.square_mesh(4, jitter=0.2, seed=1) if dim == 2 else workloads.cube_mesh(2, jitter=0.15, seed=1)
    rule = workloads.rule_for_dim(dim)
    rng = np.random.default_rng(4)
    C, V = mesh.n_cells, mesh.n_verts
    a = rng.lognormal(0, 0.5, V)
    c = np.tile(rng.uniform(0.5, 2.0, C), (rule.n_q, 1))
    A = np.zeros((V, V))
    for j in range(V):
        e = np.zeros(V)
        e[j] = 1.0
        r = ora.reaction_diffusion(mesh.coords, mesh.conn, e, a, 1, c, rule.points, rule.weights)
        np.add.at(A[:, j], mesh.conn.ravel(), r.ravel())
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    assert np.all(np.linalg.eigvalsh(0.5 * (A + A.T)) > 0)  # mass + stiffness: positive definite


# ---- the first-order term along grad a (Eq. 8: f0 depends on grad a):
#      f0 = c u + g grad a . grad u


def _linear_fields(dim, coords, seed):
    """u(x) = p.x + u0 and a(x) = s.x + a0 sampled at the vertices: exact P1 fields with
    known constant gradients p and s."""
    rng = np.random.default_rng(seed)
    p, s = rng.normal(size=dim), rng.normal(size=dim)
    u0, a0 = rng.normal(), rng.normal()
    return p @ coords + u0, s @ coords + a0, p, s


@pytest.mark.parametrize("dim", [2, 3])
def test_drift_term_closed_form(ora, dim):
    """For linear u and a the drift part is g (p.s) int_T phi_b = g (p.s) |T| / (d+1) for
    every basis function (|T| = |det J| / d!), on random, arbitrarily oriented simplices."""
    coords, conn = _random_simplices(dim, 50, 41 + dim)
    rule = workloads.rule_for_dim(dim)
    u, a, p, s = _linear_fields(dim, coords, 7 + dim)
    g = 1.7
    r_g = ora.reaction_diffusion(coords, conn, u, a, 1, None, rule.points, rule.weights, drift=g)
    r_0 = ora.reaction_diffusion(coords, conn, u, a, 1, None, rule.points, rule.weights, drift=0.0)
    X = coords.T[conn]  # [d+1][C][d]
    J = np.stack([X[j + 1] - X[0] for j in range(dim)], axis=-1)  # [C][d][d], columns x_j - x_0
    vol = np.abs(np.linalg.det(J)) / math.factorial(dim)
    want = g * float(p @ s) * vol / (dim + 1)
    d = r_g - r_0
    assert np.abs(d - want[None, :]).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_drift_term_symmetric_in_u_and_a(ora, dim):
    """grad a . grad u is symmetric, so exchanging u and a leaves the drift part unchanged
    (random nodal values: gradients differ from cell to cell)."""
    coords, conn = _random_simplices(dim, 60, 51 + dim)
    rule = workloads.rule_for_dim(dim)
    rng = np.random.default_rng(dim + 30)
    V = coords.shape[1]
    u, a = rng.uniform(-1, 1, V), rng.uniform(-1, 1, V)
    drift = lambda x, y: (ora.reaction_diffusion(coords, conn, x, y, 1, None, rule.points, rule.weights, drift=0.8)
                          - ora.reaction_diffusion(coords, conn, x, y, 1, None, rule.points, rule.weights))
    d_ua, d_au = drift(u, a), drift(a, u)
    assert np.abs(d_ua).max() > 0
    assert np.abs(d_ua - d_au).max() <= 1e-12 * np.abs(d_ua).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_drift_term_vanishes_for_p0_coefficient(ora, dim):
    """A P0 field is constant on each cell: grad a = 0 there, whatever g."""
    coords, conn = _random_simplices(dim, 20, 61 + dim)
    rule = workloads.rule_for_dim(dim)
    rng = np.random.default_rng(dim + 40)
    u, a = rng.uniform(-1, 1, coords.shape[1]), rng.lognormal(0, 1, conn.shape[1])
    c = rng.uniform(0.5, 2.0, (rule.n_q, conn.shape[1]))
    r_g = ora.reaction_diffusion(coords, conn, u, a, 0, c, rule.points, rule.weights, drift=3.0)
    r_0 = ora.reaction_diffusion(coords, conn, u, a, 0, c, rule.points, rule.weights)
    assert np.array_equal(r_g, r_0)
