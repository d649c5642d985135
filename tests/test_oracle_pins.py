"""Pins of the CPU oracle against what the weak form (Eqs. 1-2) and the mathematics fix.

Every check compares the oracle with something other than itself: closed forms,
exact simplex integrals, textbook stiffness matrices, null spaces, symmetry,
linearity identities and finite differences. A plausible mistake in the oracle (a
dropped term, a wrong sign or index, a transposed inverse Jacobian, wrong weights,
a signed determinant) fails at least one of them.
"""

import math
import os

import numpy as np
import pytest

import workloads
from workloads.meshes import Mesh, cube_mesh, square_mesh

import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_matrix(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def _tri2(ora, coords, conn, u, K=None, rule=None):
    rule = rule or workloads.rule_for_dim(coords.shape[0])
    C = conn.shape[1]
    K = np.ones((rule.n_q, C)) if K is None else K
    return ora.laplacian(coords, conn, u, K, rule.points, rule.weights)


def _random_simplices(dim, n, seed, scale=1.0):
    """n disconnected random simplices (non-degenerate), some of them negatively oriented."""
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, dim + 1, dim)) * scale
    coords = X.reshape(-1, dim).T.copy()
    conn = np.arange(n * (dim + 1), dtype=np.int32).reshape(n, dim + 1).T.copy()
    return coords, conn


# ---------------------------------------------------------------- quadrature tables


@pytest.mark.parametrize("dim", [2, 3])
def test_quadrature_rule_exact_to_degree_2(dim):
    """int over the reference simplex of xi^alpha = alpha! / (|alpha| + d)! for |alpha| <= 2."""
    rule = workloads.rule_for_dim(dim)
    assert rule.points.shape == (rule.n_q, dim)
    alphas = [a for a in np.ndindex(*(3,) * dim) if sum(a) <= 2]
    for a in alphas:
        approx = np.sum(rule.weights * np.prod(rule.points ** np.array(a), axis=1))
        want = np.prod([math.factorial(k) for k in a]) / math.factorial(sum(a) + dim)
        assert approx == pytest.approx(want, rel=1e-14, abs=1e-16), a


# ---------------------------------------------------------------- meshes


def test_mesh_sizes_and_orientation():
    m = square_mesh(64, 64, jitter=0.2, seed=0)
    assert (m.n_cells, m.n_verts) == (8192, 4225)
    assert exact.min_det(m.coords, m.conn) > 0
    m3 = cube_mesh(16, jitter=0.15, seed=0)
    assert m3.n_cells == 6 * 16 ** 3 and m3.n_verts == 17 ** 3
    assert exact.min_det(m3.coords, m3.conn) > 0
    # boundary vertices stay on the unit cube's faces
    assert m3.coords.min() == 0.0 and m3.coords.max() == 1.0


@pytest.mark.parametrize("cells", [1572864, 1 << 21])
def test_full_size_cube_meshes_positive(cells):
    n = workloads.smallest_cube_for(cells) if cells != 1 << 21 else 71
    m = cube_mesh(n, jitter=0.15, seed=0)
    m = workloads.first_cells(m, cells)
    assert m.n_cells == cells
    assert exact.min_det(m.coords, m.conn) > 0


# ---------------------------------------------------------------- closed forms


def test_reference_triangle_stiffness(ora):
    coords = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    conn = np.array([[0], [1], [2]], dtype=np.int32)
    A = np.stack([_tri2(ora, coords, conn, np.eye(3)[j])[:, 0] for j in range(3)], axis=1)
    np.testing.assert_allclose(A, _golden_matrix("reference_stiffness_tri.txt"), rtol=0, atol=1e-15)


def test_reference_tet_stiffness(ora):
    coords = np.array([[0.0, 1.0, 0.0, 0.0], [0.0, 0.0, 1.0, 0.0], [0.0, 0.0, 0.0, 1.0]])
    conn = np.array([[0], [1], [2], [3]], dtype=np.int32)
    A = np.stack([_tri2(ora, coords, conn, np.eye(4)[j])[:, 0] for j in range(4)], axis=1)
    np.testing.assert_allclose(A, _golden_matrix("reference_stiffness_tet.txt"), rtol=0, atol=1e-15)


def test_general_triangle_textbook_stiffness(ora):
    """Random (also clockwise) triangles against A_ij = (b_i b_j + c_i c_j)/(4|T|)."""
    coords, conn = _random_simplices(2, 50, seed=3)
    for c in range(conn.shape[1]):
        x = coords[:, conn[:, c]].T
        cc = coords[:, conn[:, c]]
        loc = np.arange(3, dtype=np.int32)[:, None]
        A = np.stack([_tri2(ora, cc, loc, np.eye(3)[j])[:, 0] for j in range(3)], axis=1)
        np.testing.assert_allclose(A, exact.triangle_stiffness(x), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_scaling_covariance(ora, dim):
    """A cell scaled by s gives s^(d-2) times the Laplacian element vector."""
    coords, conn = _random_simplices(dim, 20, seed=5)
    u = np.random.default_rng(1).uniform(-1, 1, coords.shape[1])
    r1 = _tri2(ora, coords, conn, u)
    for s in (0.01, 3.0):
        rs = _tri2(ora, s * coords, conn, u)
        np.testing.assert_allclose(rs, s ** (dim - 2) * r1, rtol=1e-12, atol=1e-14 * np.abs(r1).max())


# ---------------------------------------------------------------- exact integration, polynomial K


def _poly(dim, seed):
    rng = np.random.default_rng(seed)
    g = rng.uniform(-1, 1, dim)
    H = rng.uniform(-1, 1, (dim, dim))
    return 2.5, g, 0.5 * (H + H.T)


def _quad_points(coords, conn, rule):
    bary = np.concatenate([1.0 - rule.points.sum(1, keepdims=True), rule.points], axis=1)
    return np.einsum("qb,ibc->qic", bary, coords[:, conn])


@pytest.mark.parametrize("dim", [2, 3])
def test_polynomial_K_exact_on_distorted_mesh(ora, dim):
    """Degree-2 K sampled at the quadrature points: the degree-2 rule integrates it
    exactly, so r_b = (int_T K) grad phi_b . grad u with exact simplex moments."""
    mesh = square_mesh(6, 5, jitter=0.3, seed=11) if dim == 2 else cube_mesh(3, jitter=0.2, seed=11)
    rule = workloads.rule_for_dim(dim)
    k0, g, H = _poly(dim, 2)
    K = exact.quadratic_at(_quad_points(mesh.coords, mesh.conn, rule), k0, g, H)
    u = np.random.default_rng(4).uniform(-1, 1, mesh.n_verts)
    r = ora.laplacian(mesh.coords, mesh.conn, u, K, rule.points, rule.weights)
    want = exact.laplacian_exact(mesh.coords, mesh.conn, u,
                                 exact.quadratic_integral(mesh.coords, mesh.conn, k0, g, H))
    np.testing.assert_allclose(r, want, rtol=0, atol=1e-13 * np.abs(want).max())


@pytest.mark.parametrize("dim", [2, 3])
def test_polynomial_K_exact_random_orientation(ora, dim):
    """Same on isolated random simplices, half of them negatively oriented: pins |det J|."""
    coords, conn = _random_simplices(dim, 40, seed=21)
    rule = workloads.rule_for_dim(dim)
    k0, g, H = _poly(dim, 8)
    k0 = 40.0  # keep K > 0 on the random cells
    K = exact.quadratic_at(_quad_points(coords, conn, rule), k0, g, H)
    u = np.random.default_rng(5).uniform(-1, 1, coords.shape[1])
    r = ora.laplacian(coords, conn, u, K, rule.points, rule.weights)
    want = exact.laplacian_exact(coords, conn, u, exact.quadratic_integral(coords, conn, k0, g, H))
    assert exact.min_det(coords, conn) < 0  # the case is really exercised
    np.testing.assert_allclose(r, want, rtol=0, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("dim", [2, 3])
def test_elasticity_polynomial_lame_exact(ora, dim):
    mesh = square_mesh(5, 4, jitter=0.3, seed=12) if dim == 2 else cube_mesh(2, jitter=0.2, seed=12)
    rule = workloads.rule_for_dim(dim)
    xq = _quad_points(mesh.coords, mesh.conn, rule)
    pl, pm = _poly(dim, 6), _poly(dim, 7)
    lam = exact.quadratic_at(xq, *pl)
    mu = exact.quadratic_at(xq, *pm)
    u = np.random.default_rng(9).normal(0, 1e-2, (dim, mesh.n_verts))
    r = ora.elasticity(mesh.coords, mesh.conn, u, lam, mu, rule.points, rule.weights)
    want = exact.elasticity_exact(mesh.coords, mesh.conn, u,
                                  exact.quadratic_integral(mesh.coords, mesh.conn, *pl),
                                  exact.quadratic_integral(mesh.coords, mesh.conn, *pm))
    np.testing.assert_allclose(r, want, rtol=0, atol=1e-13 * np.abs(want).max())


# ---------------------------------------------------------------- null spaces and invariants


@pytest.mark.parametrize("dim", [2, 3])
def test_constant_field_gives_zero(ora, dim):
    case = workloads.laplacian_square_case(16) if dim == 2 else workloads.laplacian_cube_case(6 * 6 ** 3)
    u = np.full(case.n_verts, 0.7)
    r = ora.laplacian(case.mesh.coords, case.mesh.conn, u, case.K, case.rule.points, case.rule.weights)
    scale = np.abs(ora.residual_for(case)).max()
    assert np.abs(r).max() <= 1e-14 * max(scale, 1.0)


@pytest.mark.parametrize("dim", [2, 3])
def test_rigid_motions_give_zero(ora, dim):
    case = workloads.elasticity_case(dim, 2 * 8 * 8 if dim == 2 else 6 * 4 ** 3)
    x = case.mesh.coords
    rng = np.random.default_rng(0)
    a = rng.normal(size=dim)
    if dim == 2:
        w = 0.3
        u = a[:, None] + w * np.stack([-x[1], x[0]])
    else:
        w = rng.normal(size=3)
        u = a[:, None] + np.cross(w, x.T).T
    r = ora.elasticity(x, case.mesh.conn, u, case.lam, case.mu, case.rule.points, case.rule.weights)
    scale = np.abs(ora.elasticity(x, case.mesh.conn, case.u * 100, case.lam, case.mu,
                                  case.rule.points, case.rule.weights)).max()
    assert np.abs(r).max() <= 1e-13 * scale


@pytest.mark.parametrize("dim", [2, 3])
def test_element_sums_vanish(ora, dim):
    case = workloads.laplacian_square_case(16) if dim == 2 else workloads.laplacian_cube_case(6 * 5 ** 3)
    r = ora.residual_for(case)
    assert np.abs(r.sum(axis=0)).max() <= 1e-14 * np.abs(r).max()
    e = workloads.elasticity_case(dim, 128 if dim == 2 else 6 * 3 ** 3)
    re = ora.residual_for(e)
    per_comp = re.reshape(dim + 1, dim, -1).sum(axis=0)
    assert np.abs(per_comp).max() <= 1e-14 * np.abs(re).max()


def _assembled_operator(conn, V, elem_fn, n_comp):
    n = V * n_comp
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = exact.assemble(conn, elem_fn(e.reshape(n_comp, V)), V, n_comp).ravel()
    return A


@pytest.mark.parametrize("dim", [2, 3])
def test_assembled_laplacian_symmetric_and_patch(ora, dim):
    case = workloads.laplacian_square_case(6) if dim == 2 else workloads.laplacian_cube_case(6 * 3 ** 3)
    m, q = case.mesh, case.rule
    fn = lambda U: ora.laplacian(m.coords, m.conn, U[0], case.K, q.points, q.weights)
    A = _assembled_operator(m.conn, m.n_verts, fn, 1)
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    # patch test: linear u and constant K give a zero assembled residual at interior nodes
    lin = 0.3 + np.array([1.0, -2.0, 0.5][:dim]) @ m.coords
    K1 = np.full_like(case.K, 1.7)
    R = exact.assemble(m.conn, ora.laplacian(m.coords, m.conn, lin, K1, q.points, q.weights), m.n_verts)[0]
    interior = np.all((m.coords > 1e-12) & (m.coords < 1 - 1e-12), axis=0)
    assert interior.any()
    assert np.abs(R[interior]).max() <= 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_assembled_elasticity_symmetric(ora, dim):
    case = workloads.elasticity_case(dim, 2 * 4 * 4 if dim == 2 else 6 * 2 ** 3)
    m, q = case.mesh, case.rule
    fn = lambda U: ora.elasticity(m.coords, m.conn, U, case.lam, case.mu, q.points, q.weights)
    A = _assembled_operator(m.conn, m.n_verts, fn, dim)
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_assembled_elasticity_patch(ora, dim):
    """Patch test: a linear displacement u = A x + b with constant lambda, mu has a constant
    stress, so the assembled residual vanishes at every interior vertex."""
    case = workloads.elasticity_case(dim, 2 * 6 * 6 if dim == 2 else 6 * 3 ** 3)
    m, q = case.mesh, case.rule
    rng = np.random.default_rng(dim + 11)
    A = rng.normal(size=(dim, dim))
    b = rng.normal(size=dim)
    U = A @ m.coords + b[:, None]
    lam = np.full_like(case.lam, 1.3)
    mu = np.full_like(case.mu, 0.7)
    R = exact.assemble(m.conn, ora.elasticity(m.coords, m.conn, U, lam, mu, q.points, q.weights), m.n_verts, dim)
    interior = np.all((m.coords > 1e-12) & (m.coords < 1 - 1e-12), axis=0)
    assert interior.any()
    scale = np.abs(ora.elasticity(m.coords, m.conn, U, lam, mu, q.points, q.weights)).max()
    assert np.abs(R[:, interior]).max() <= 1e-13 * scale


def test_paper_listings_special_cases(ora):
    """K = 1 is the Laplacian listing (f1 = grad u); lambda = 0, mu = 1/2 is the 2D
    elasticity listing (f1 = symmetric gradient), both from Sec. 6."""
    mesh = square_mesh(4, 3, jitter=0.25, seed=2)
    rule = workloads.triangle_deg2()
    C = mesh.n_cells
    u2 = np.random.default_rng(3).normal(size=(2, mesh.n_verts))
    zero = np.zeros((rule.n_q, C))
    half = np.full((rule.n_q, C), 0.5)
    r = ora.elasticity(mesh.coords, mesh.conn, u2, zero, half, rule.points, rule.weights)
    G, vol = exact.p1_gradients(mesh.coords, mesh.conn)
    ub = np.transpose(u2[:, mesh.conn], (2, 1, 0))  # (C, b, k)
    gradu = np.einsum("cbk,cbi->cki", ub, G)
    f1 = 0.5 * (gradu + np.transpose(gradu, (0, 2, 1)))  # the listing's f1 per component
    want = np.einsum("c,cki,cbi->cbk", vol, f1, G).reshape(C, -1).T
    np.testing.assert_allclose(r, want, rtol=0, atol=1e-13 * np.abs(want).max())
    u1 = u2[0]
    r1 = ora.laplacian(mesh.coords, mesh.conn, u1, np.ones((rule.n_q, C)), rule.points, rule.weights)
    want1 = exact.laplacian_exact(mesh.coords, mesh.conn, u1, vol)
    np.testing.assert_allclose(r1, want1, rtol=0, atol=1e-13 * np.abs(want1).max())


# ---------------------------------------------------------------- adjoint


def _J(ora, case, u, K, lam):
    m, q = case.mesh, case.rule
    return float(np.sum(lam * ora.laplacian(m.coords, m.conn, u, K, q.points, q.weights)))


@pytest.mark.parametrize("dim", [2, 3])
def test_adjoint_linearity_identities(ora, dim):
    """J is linear in u and in K separately, so J = dJ/du . u = dJ/dK : K exactly."""
    case = workloads.laplacian_square_case(8) if dim == 2 else workloads.laplacian_cube_case(6 * 4 ** 3)
    lam = np.random.default_rng(17).uniform(-1, 1, (dim + 1, case.n_cells))
    dK, du = ora.adjoint_for(case, lam)
    J = _J(ora, case, case.u, case.K, lam)
    assert float(du @ case.u) == pytest.approx(J, rel=1e-12)
    assert float(np.sum(dK * case.K)) == pytest.approx(J, rel=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_adjoint_central_differences(ora, dim):
    """Central differences with h = 1e-6 in 64 random directions (seeds 1..64)."""
    case = workloads.laplacian_square_case(6) if dim == 2 else workloads.laplacian_cube_case(6 * 3 ** 3)
    lam = np.random.default_rng(23).uniform(-1, 1, (dim + 1, case.n_cells))
    dK, du = ora.adjoint_for(case, lam)
    h = 1e-6
    for s in range(1, 65):
        rng = np.random.default_rng(s)
        dKdir = rng.normal(size=case.K.shape)
        dudir = rng.normal(size=case.u.shape)
        fdK = (_J(ora, case, case.u, case.K + h * dKdir, lam) - _J(ora, case, case.u, case.K - h * dKdir, lam)) / (2 * h)
        fdu = (_J(ora, case, case.u + h * dudir, case.K, lam) - _J(ora, case, case.u - h * dudir, case.K, lam)) / (2 * h)
        assert fdK == pytest.approx(np.sum(dK * dKdir), rel=1e-7, abs=1e-9)
        assert fdu == pytest.approx(du @ dudir, rel=1e-7, abs=1e-9)


def test_adjoint_element_gradient_is_stiffness_transpose(ora):
    """dJ/du on a single cell equals A_e^T lambda with the textbook triangle stiffness."""
    coords, conn = _random_simplices(2, 1, seed=31)
    rule = workloads.triangle_deg2()
    K = np.full((3, 1), 2.0)
    lam = np.array([[0.3], [-1.1], [0.5]])
    u = np.array([0.2, 0.9, -0.4])
    dK, du = ora.adjoint_laplacian(coords, conn, u, K, rule.points, rule.weights, lam)
    A = 2.0 * exact.triangle_stiffness(coords[:, conn[:, 0]].T)
    np.testing.assert_allclose(du, A.T @ lam[:, 0], rtol=1e-12)


def test_oracle_errors(ora):
    from oracle import OracleError

    coords = np.zeros((2, 3))
    conn = np.array([[0], [1], [5]], dtype=np.int32)
    rule = workloads.triangle_deg2()
    with pytest.raises(OracleError):
        ora.laplacian(coords, conn, np.zeros(3), np.ones((3, 1)), rule.points, rule.weights)
    conn = np.array([[0], [1], [2]], dtype=np.int32)
    with pytest.raises(OracleError):  # degenerate cell
        ora.laplacian(coords, conn, np.zeros(3), np.ones((3, 1)), rule.points, rule.weights)
    empty = ora.laplacian(coords, np.zeros((3, 0), np.int32), np.zeros(3), np.ones((3, 0)),
                          rule.points, rule.weights)
    assert empty.shape == (3, 0)


@pytest.mark.parametrize("dim", [2, 3])
def test_adjoint_random_orientation_differences(ora, dim):
    """Central differences on isolated random simplices, some negatively oriented (pins
    |det J| in the adjoint too)."""
    coords, conn = _random_simplices(dim, 12, seed=41)
    assert exact.min_det(coords, conn) < 0
    rule = workloads.rule_for_dim(dim)
    rng = np.random.default_rng(2)
    C, V = conn.shape[1], coords.shape[1]
    K = rng.lognormal(0, 1, (rule.n_q, C))
    u = rng.uniform(-1, 1, V)
    lam = rng.uniform(-1, 1, (dim + 1, C))
    dK, du = ora.adjoint_laplacian(coords, conn, u, K, rule.points, rule.weights, lam)
    J = lambda uu, KK: float(np.sum(lam * ora.laplacian(coords, conn, uu, KK, rule.points, rule.weights)))
    h = 1e-6
    for s in range(8):
        r2 = np.random.default_rng(100 + s)
        dKd, dud = r2.normal(size=K.shape), r2.normal(size=V)
        assert (J(u, K + h * dKd) - J(u, K - h * dKd)) / (2 * h) == pytest.approx(np.sum(dK * dKd), rel=1e-7)
        assert (J(u + h * dud, K) - J(u - h * dud, K)) / (2 * h) == pytest.approx(du @ dud, rel=1e-7)
