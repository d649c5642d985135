"""Pins of the oracle's pointwise-physics routine (Eq. 2, both terms, for pointwise
functions f0 and f1 chosen by the caller; the library compiles them from source strings
at run time, Sec. 5): the Laplacian and Lame choices reproduce the already pinned
Laplacian and elasticity routines; the reaction choice gives the closed-form P1 mass
matrix plus the exact source integral; the nonlinear coefficient kappa(u, x) grad u of
Sec. 2 is integrated exactly by the degree-2 rule whenever kappa(u(x), x) is a polynomial
of degree <= 2 in x (u is linear on a P1 cell), against the exact simplex moments
int lambda_a lambda_b = |T| (1 + delta_ab) / ((d+1)(d+2)); a constant field gives zero."""

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


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_laplacian_choice_is_the_laplacian_routine(ora, dim):
    coords, conn = _random_simplices(dim, 60, dim)
    rule = workloads.rule_for_dim(dim)
    rng = np.random.default_rng(1)
    u = rng.uniform(-1, 1, coords.shape[1])
    K = rng.lognormal(0, 1, (rule.n_q, conn.shape[1]))
    r = ora.pointwise("laplacian", coords, conn, u, K[None], rule.points, rule.weights)
    assert _rel(r, ora.laplacian(coords, conn, u, K, rule.points, rule.weights)) <= 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_lame_choice_is_the_elasticity_routine(ora, dim):
    coords, conn = _random_simplices(dim, 60, 10 + dim)
    rule = workloads.rule_for_dim(dim)
    rng = np.random.default_rng(2)
    u = rng.normal(0, 1, (dim, coords.shape[1]))
    lam = rng.lognormal(0, 0.5, (rule.n_q, conn.shape[1]))
    mu = rng.lognormal(0, 0.5, (rule.n_q, conn.shape[1]))
    r = ora.pointwise("elasticity", coords, conn, u, np.stack([lam, mu]), rule.points, rule.weights)
    assert _rel(r, ora.elasticity(coords, conn, u, lam, mu, rule.points, rule.weights)) <= 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_reaction_choice_mass_matrix_and_source(ora, dim):
    """f0 = a0 u + p0 with a constant a0 and no diffusion: r_b = a0 sum_a M_ba u_a + p0 |T|/(d+1),
    M_ba = |T| (1 + delta_ab) / ((d+1)(d+2))."""
    coords, conn = _random_simplices(dim, 50, 20 + dim)
    rule = workloads.rule_for_dim(dim)
    C, nb = conn.shape[1], dim + 1
    rng = np.random.default_rng(3)
    u = rng.uniform(-1, 1, coords.shape[1])
    a0, p0 = 1.7, -0.4
    coef = np.stack([np.full((rule.n_q, C), a0), np.zeros((rule.n_q, C))])
    r = ora.pointwise("reaction", coords, conn, u, coef, rule.points, rule.weights, params=(p0, 0, 0, 0))
    _, vol = exact.p1_gradients(coords, conn)
    ub = u[conn]  # (b, C)
    mass = vol / ((dim + 1) * (dim + 2)) * (ub + ub.sum(axis=0))  # sum_a M_ba u_a
    ref = a0 * mass + p0 * vol / nb
    assert _rel(r, ref) <= 1e-13


def _grad_terms(coords, conn, u):
    G, vol = exact.p1_gradients(coords, conn)
    g = np.einsum("cb,cbi->ci", u[conn].T, G)
    return np.einsum("cbi,ci->bc", G, g), vol  # G_b . g per (b, cell)


@pytest.mark.parametrize("dim", [2, 3])
def test_nonlinear_kappa_of_u_exact(ora, dim):
    """kappa = p0 + p1 u + p2 u^2 with u linear on the cell: r_b = (G_b . g) int_T kappa(u),
    int u = |T| mean(u_b), int u^2 = |T| ((sum u_b)^2 + sum u_b^2) / ((d+1)(d+2))."""
    coords, conn = _random_simplices(dim, 80, 30 + dim)
    rule = workloads.rule_for_dim(dim)
    u = np.random.default_rng(4).uniform(-1, 1, coords.shape[1])
    p = (1.3, -0.7, 0.45, 0.0)
    r = ora.pointwise("nonlinear", coords, conn, u, None, rule.points, rule.weights, params=p)
    gg, vol = _grad_terms(coords, conn, u)
    ub = u[conn]
    s1, s2 = ub.sum(axis=0), (ub ** 2).sum(axis=0)
    int_kappa = vol * (p[0] + p[1] * s1 / (dim + 1) + p[2] * (s1 ** 2 + s2) / ((dim + 1) * (dim + 2)))
    assert _rel(r, gg * int_kappa) <= 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_nonlinear_kappa_of_u_and_x_exact(ora, dim):
    """kappa = (p0 + p1 u)(1 + p3 s(x)), s = x_0 + 2 x_1 (+ 3 x_2): degree 2 in x, so the rule
    is exact; with s linear, int u s = |T| ((sum u_b)(sum s_b) + sum u_b s_b) / ((d+1)(d+2)),
    int s = |T| mean(s_b)."""
    coords, conn = _random_simplices(dim, 80, 40 + dim)
    rule = workloads.rule_for_dim(dim)
    u = np.random.default_rng(6).uniform(-1, 1, coords.shape[1])
    p = (0.8, 1.1, 0.0, -0.6)
    r = ora.pointwise("nonlinear", coords, conn, u, None, rule.points, rule.weights, params=p)
    gg, vol = _grad_terms(coords, conn, u)
    s_vert = (np.arange(1, dim + 1)[:, None] * coords).sum(axis=0)  # s at the vertices
    ub, xb = u[conn], s_vert[conn]
    su, sx = ub.sum(axis=0), xb.sum(axis=0)
    k = (dim + 1) * (dim + 2)
    int_kappa = vol * (p[0] + p[0] * p[3] * sx / (dim + 1) + p[1] * su / (dim + 1)
                       + p[1] * p[3] * (su * sx + (ub * xb).sum(axis=0)) / k)
    assert _rel(r, gg * int_kappa) <= 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_nonlinear_constant_field_gives_zero(ora, dim):
    coords, conn = _random_simplices(dim, 30, 50 + dim)
    rule = workloads.rule_for_dim(dim)
    p = (1.0, 2.0, 3.0, 0.5)
    u = np.full(coords.shape[1], 0.8)
    r = ora.pointwise("nonlinear", coords, conn, u, None, rule.points, rule.weights, params=p)
    # rounding only: against the size of the residual of a field of the same magnitude
    v = np.random.default_rng(7).uniform(-0.8, 0.8, coords.shape[1])
    scale = np.abs(ora.pointwise("nonlinear", coords, conn, v, None, rule.points, rule.weights, params=p)).max()
    assert np.abs(r).max() <= 1e-13 * scale


def test_pointwise_argument_checks(ora):
    coords, conn = _random_simplices(3, 4, 1)
    rule = workloads.rule_for_dim(3)
    u = np.zeros(coords.shape[1])
    with pytest.raises(ora.OracleError):  # the Laplacian choice needs one coefficient
        ora.pointwise("laplacian", coords, conn, u, None, rule.points, rule.weights)
    with pytest.raises(ora.OracleError):  # Lame needs dim components
        ora.pointwise("elasticity", coords, conn, u, np.zeros((2, rule.n_q, 4)), rule.points, rule.weights)
