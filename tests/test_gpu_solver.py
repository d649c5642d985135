"""The matrix-free Jacobi-preconditioned CG solve with the assembled Laplacian (Eq. 2:
E^T of the element residuals), against the patch test (a linear field is the exact
discrete solution for a constant coefficient) and against a dense direct solve of the
operator assembled from the CPU oracle's element vectors."""

import numpy as np
import pytest
import torch

import oracle
import paper_1607_04245_gb300 as fem
import workloads
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _mesh(dim, n):
    return workloads.square_mesh(n, jitter=0.2, seed=3) if dim == 2 else workloads.cube_mesh(n, jitter=0.15, seed=3)


def _boundary(mesh):
    x = mesh.coords
    return np.any((np.abs(x) < 1e-14) | (np.abs(x - 1.0) < 1e-14), axis=0)


def _oracle_operator(mesh, K, rule):
    V = mesh.n_verts
    A = np.zeros((V, V))
    for j in range(V):
        e = np.zeros(V)
        e[j] = 1.0
        r = oracle.laplacian(mesh.coords, mesh.conn, e, K, rule.points, rule.weights)
        np.add.at(A[:, j], mesh.conn.ravel(), r.ravel())
    return A


def _solve(mesh, K, rule, fixed, x0, b, prec, rtol):
    dt = fem.value_dtype(prec)
    coords, conn = to_dev(mesh.coords, torch.float64), to_dev(mesh.conn, torch.int32)
    ptr, idx = fem.fem_build_node2cell(conn, mesh.n_verts)
    x = to_dev(x0, dt)
    return fem.fem_pcg_laplacian(coords, conn, to_dev(K, dt), rule.points, rule.weights, ptr, idx,
                                 to_dev(fixed.astype(np.uint8), torch.uint8), x,
                                 b=None if b is None else to_dev(b, dt), max_iter=5000, rtol=rtol, prec=prec)


@pytest.mark.parametrize("dim,n", [(2, 24), (3, 8)])
def test_patch_test_linear_solution(dim, n):
    mesh = _mesh(dim, n)
    rule = workloads.rule_for_dim(dim)
    K = np.full((rule.n_q, mesh.n_cells), 1.7)
    coef = np.array([1.0, 2.0, -3.0, 0.5][: dim + 1])
    g = coef[0] + coef[1:] @ mesh.coords
    fixed = _boundary(mesh)
    x0 = np.where(fixed, g, 0.0)
    x, iters, resid = _solve(mesh, K, rule, fixed, x0, None, "fp64", 1e-13)
    err = np.abs(x.cpu().numpy() - g).max() / np.abs(g).max()
    assert resid <= 1e-13 and iters > 0
    assert err <= 1e-10, err


@pytest.mark.parametrize("dim,n", [(2, 12), (3, 4)])
@pytest.mark.parametrize("prec,rtol,tol", [("fp64", 1e-12, 1e-9), ("fp64_df", 1e-12, 1e-9), ("mixed", 1e-5, 1e-4)])
def test_matches_dense_solve_of_oracle_operator(dim, n, prec, rtol, tol):
    mesh = _mesh(dim, n)
    rule = workloads.rule_for_dim(dim)
    rng = np.random.default_rng(dim)
    K = rng.lognormal(0.0, 1.0, (rule.n_q, mesh.n_cells))
    if prec == "mixed":
        K = K.astype(np.float32).astype(np.float64)
    fixed = _boundary(mesh)
    g = np.sin(mesh.coords[0] * 3.0) + mesh.coords[1]
    b = np.where(fixed, 0.0, rng.uniform(-1, 1, mesh.n_verts) / mesh.n_verts)
    if prec == "mixed":
        b = b.astype(np.float32).astype(np.float64)
        g = g.astype(np.float32).astype(np.float64)
    x0 = np.where(fixed, g, 0.0)
    x, iters, resid = _solve(mesh, K, rule, fixed, x0, b, prec, rtol)
    A = _oracle_operator(mesh, K, rule)
    free = ~fixed
    ref = x0.copy()
    ref[free] = np.linalg.solve(A[np.ix_(free, free)], b[free] - A[np.ix_(free, fixed)] @ g[fixed])
    err = np.abs(x.cpu().numpy().astype(np.float64) - ref).max() / np.abs(ref).max()
    assert resid <= rtol
    assert err <= tol, (err, iters, resid)


def test_solve_is_reproducible():
    mesh = _mesh(2, 16)
    rule = workloads.rule_for_dim(2)
    K = np.random.default_rng(1).lognormal(0.0, 1.0, (rule.n_q, mesh.n_cells))
    fixed = _boundary(mesh)
    x0 = np.where(fixed, mesh.coords[0], 0.0)
    a = _solve(mesh, K, rule, fixed, x0, None, "fp64", 1e-10)[0].cpu().numpy()
    b = _solve(mesh, K, rule, fixed, x0, None, "fp64", 1e-10)[0].cpu().numpy()
    assert np.array_equal(a, b)


def test_workspace_too_small_is_rejected():
    mesh = _mesh(2, 4)
    rule = workloads.rule_for_dim(2)
    coords, conn = to_dev(mesh.coords, torch.float64), to_dev(mesh.conn, torch.int32)
    ptr, idx = fem.fem_build_node2cell(conn, mesh.n_verts)
    K = torch.ones((rule.n_q, mesh.n_cells), dtype=torch.float64, device="cuda")
    fixed = torch.zeros(mesh.n_verts, dtype=torch.uint8, device="cuda")
    x = torch.zeros(mesh.n_verts, dtype=torch.float64, device="cuda")
    with pytest.raises(fem.FemError):
        fem.fem_pcg_laplacian(coords, conn, K, rule.points, rule.weights, ptr, idx, fixed, x,
                              work=torch.empty(16, dtype=torch.uint8, device="cuda"), prec="fp64")


def test_double_float_residual_solves_like_float64():
    """The solve with the double-float residual (float64 values, 4e-14 residual error)
    takes the float64 solve's path: same iteration count to within a few, same solution
    to 1e-10 on the 3D workload mesh's first 24^3 x 6 cells."""
    mesh = _mesh(3, 24)
    rule = workloads.rule_for_dim(3)
    K = np.random.default_rng(5).lognormal(0.0, 1.0, (rule.n_q, mesh.n_cells))
    fixed = _boundary(mesh)
    x0 = np.where(fixed, 1.0 + 2.0 * mesh.coords[0] - 3.0 * mesh.coords[1], 0.0)
    x64, it64, r64 = _solve(mesh, K, rule, fixed, x0, None, "fp64", 1e-10)
    xdf, itdf, rdf = _solve(mesh, K, rule, fixed, x0, None, "fp64_df", 1e-10)
    assert r64 <= 1e-10 and rdf <= 1e-10
    assert abs(it64 - itdf) <= 3, (it64, itdf)
    a, b = x64.cpu().numpy(), xdf.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max()


def test_concurrent_solves_from_two_threads():
    """Two host threads solving on their own streams get the single-threaded results
    (the loop captures are serialised inside the library)."""
    import threading

    mesh = _mesh(2, 16)
    rule = workloads.rule_for_dim(2)
    K = np.random.default_rng(2).lognormal(0.0, 1.0, (rule.n_q, mesh.n_cells))
    fixed = _boundary(mesh)
    x0 = np.where(fixed, mesh.coords[0] - mesh.coords[1], 0.0)
    ref = _solve(mesh, K, rule, fixed, x0, None, "fp64", 1e-10)[0].cpu().numpy()
    results, errors = [None, None], []

    def worker(i):
        try:
            with torch.cuda.stream(torch.cuda.Stream()):
                s = torch.cuda.current_stream()
                coords, conn = to_dev(mesh.coords, torch.float64), to_dev(mesh.conn, torch.int32)
                ptr, idx = fem.fem_build_node2cell(conn, mesh.n_verts, stream=s)
                x = to_dev(x0, torch.float64)
                for _ in range(3):
                    x.copy_(to_dev(x0, torch.float64))
                    fem.fem_pcg_laplacian(coords, conn, to_dev(K, torch.float64), rule.points, rule.weights, ptr, idx,
                                          to_dev(fixed.astype(np.uint8), torch.uint8), x, max_iter=5000, rtol=1e-10,
                                          prec="fp64", stream=s)
                s.synchronize()
                results[i] = x.cpu().numpy()
        except Exception as exc:  # reported below
            errors.append(exc)

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for r in results:
        assert np.array_equal(r, ref)


def _solve_refined(mesh, K, rule, fixed, x0, b, rtol, residual_prec="fp64", inner_rtol=1e-3):
    coords, conn = to_dev(mesh.coords, torch.float64), to_dev(mesh.conn, torch.int32)
    ptr, idx = fem.fem_build_node2cell(conn, mesh.n_verts)
    x = to_dev(x0, torch.float64)
    return fem.fem_pcg_laplacian_refined(coords, conn, to_dev(K, torch.float64), rule.points, rule.weights, ptr, idx,
                                         to_dev(fixed.astype(np.uint8), torch.uint8), x,
                                         b=None if b is None else to_dev(b, torch.float64), max_outer=30,
                                         max_inner=5000, inner_rtol=inner_rtol, rtol=rtol,
                                         residual_prec=residual_prec)


@pytest.mark.parametrize("dim,n", [(2, 12), (3, 4)])
@pytest.mark.parametrize("residual_prec", ["fp64", "fp64_df"])
def test_refined_solve_matches_dense_solve_of_oracle_operator(dim, n, residual_prec):
    """Mixed-precision iterative refinement (float32-mixed corrections, float64 residuals)
    reaches the float64 solution: against a dense solve of the operator assembled from the
    oracle's element vectors, at the float64 solve's tolerance, with float64 inputs."""
    mesh = _mesh(dim, n)
    rule = workloads.rule_for_dim(dim)
    rng = np.random.default_rng(dim + 10)
    K = rng.lognormal(0.0, 1.0, (rule.n_q, mesh.n_cells))
    fixed = _boundary(mesh)
    g = np.sin(mesh.coords[0] * 3.0) + mesh.coords[1]
    b = np.where(fixed, 0.0, rng.uniform(-1, 1, mesh.n_verts) / mesh.n_verts)
    x0 = np.where(fixed, g, 0.0)
    x, outer, inner, resid = _solve_refined(mesh, K, rule, fixed, x0, b, 1e-12, residual_prec)
    A = _oracle_operator(mesh, K, rule)
    free = ~fixed
    ref = x0.copy()
    ref[free] = np.linalg.solve(A[np.ix_(free, free)], b[free] - A[np.ix_(free, fixed)] @ g[fixed])
    err = np.abs(x.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert resid <= 1e-12 and outer >= 2 and inner > 0
    assert err <= 1e-9, (err, outer, inner, resid)
    # the residual of the returned x recomputed from the oracle's operator
    r = np.where(free, b - A @ x.cpu().numpy(), 0.0)
    r0 = np.where(free, b - A @ x0, 0.0)
    assert np.linalg.norm(r) <= 2e-12 * np.linalg.norm(r0)


def test_refined_solve_full_mesh_agrees_with_float64_pcg():
    """On the 1,572,864-tet workload mesh: the refined solve to 1e-8 and the float64 PCG to
    1e-8 give the same solution to the accuracy the tolerance allows, the refinement in a few
    outer steps; the Dirichlet values are kept."""
    case = workloads.laplacian_cube_case()
    mesh, rule = case.mesh, case.rule
    fixed, x0 = workloads.cases.dirichlet_problem(case)
    fixed = fixed.astype(bool)
    x64, it64, r64 = _solve(mesh, case.K, rule, fixed, x0, None, "fp64", 1e-8)
    xr, outer, inner, rr = _solve_refined(mesh, case.K, rule, fixed, x0, None, 1e-8)
    assert r64 <= 1e-8 and rr <= 1e-8
    assert 1 <= outer <= 6, (outer, inner)
    a, b = x64.cpu().numpy(), xr.cpu().numpy()
    assert np.array_equal(b[fixed], x0[fixed])
    assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max(), (np.abs(a - b).max(), outer, inner)


@pytest.mark.parametrize("dim,n", [(2, 16), (3, 6)])
def test_iterations_match_textbook_pcg_on_oracle_operator(dim, n):
    """The device loop (Chronopoulos and Gear's form of CG: one reduction per iteration)
    against the textbook Jacobi-PCG written out in numpy on the operator assembled from the
    oracle's element vectors: the same iteration count to within 2 and the same solution."""
    mesh = _mesh(dim, n)
    rule = workloads.rule_for_dim(dim)
    rng = np.random.default_rng(dim + 20)
    K = rng.lognormal(0.0, 1.0, (rule.n_q, mesh.n_cells))
    fixed = _boundary(mesh)
    g = 1.0 + mesh.coords[0] - 2.0 * mesh.coords[1]
    b = np.where(fixed, 0.0, rng.uniform(-1, 1, mesh.n_verts) / mesh.n_verts)
    x0 = np.where(fixed, g, 0.0)
    rtol = 1e-10
    x, iters, resid = _solve(mesh, K, rule, fixed, x0, b, "fp64", rtol)
    A = _oracle_operator(mesh, K, rule)
    free = ~fixed
    Af = A[np.ix_(free, free)]
    rhs = b[free] - A[np.ix_(free, fixed)] @ x0[fixed]
    d = np.diag(Af)
    xf = np.zeros(free.sum())
    r = rhs - Af @ xf
    z = r / d
    p = z.copy()
    rz = r @ z
    r0 = np.linalg.norm(r)
    k = 0
    while np.linalg.norm(r) > rtol * r0 and k < 5000:
        q = Af @ p
        alpha = rz / (p @ q)
        xf += alpha * p
        r -= alpha * q
        z = r / d
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        k += 1
    ref = x0.copy()
    ref[free] = xf
    assert abs(iters - k) <= 2, (iters, k)
    assert resid <= rtol
    assert np.abs(x.cpu().numpy() - ref).max() <= 1e-8 * np.abs(ref).max()


def _oracle_elasticity_operator(mesh, lam, mu, rule):
    """Dense assembled elasticity operator ([dim][V] unknowns, component-major) by probing
    the oracle's element residuals with unit displacements."""
    dim, V = mesh.dim, mesh.n_verts
    N = dim * V
    A = np.zeros((N, N))
    for j in range(N):
        u = np.zeros((dim, V))
        u[j // V, j % V] = 1.0
        r = oracle.elasticity(mesh.coords, mesh.conn, u, lam, mu, rule.points, rule.weights)
        for a in range(dim + 1):
            for k in range(dim):
                np.add.at(A[k * V:(k + 1) * V, j], mesh.conn[a], r[a * dim + k])
    return A


def _solve_el(mesh, lam, mu, rule, fixed, x0, b, prec, rtol):
    dt = fem.value_dtype(prec)
    coords, conn = to_dev(mesh.coords, torch.float64), to_dev(mesh.conn, torch.int32)
    ptr, idx = fem.fem_build_node2cell(conn, mesh.n_verts)
    x = to_dev(x0, dt)
    return fem.fem_pcg_elasticity(coords, conn, to_dev(lam, dt), to_dev(mu, dt), rule.points, rule.weights, ptr, idx,
                                  to_dev(fixed.astype(np.uint8), torch.uint8), x,
                                  b=None if b is None else to_dev(b, dt), max_iter=20000, rtol=rtol, prec=prec)


@pytest.mark.parametrize("dim,n", [(2, 16), (3, 5)])
def test_elasticity_patch_test_linear_solution(dim, n):
    """Constant Lame parameters and a linear displacement held on the boundary: the linear
    field is the exact discrete solution (patch test)."""
    mesh = _mesh(dim, n)
    rule = workloads.rule_for_dim(dim)
    lam = np.full((rule.n_q, mesh.n_cells), 1.3)
    mu = np.full((rule.n_q, mesh.n_cells), 0.7)
    Amat = np.arange(1, dim * dim + 1, dtype=np.float64).reshape(dim, dim) / 10.0
    g = Amat @ mesh.coords + 0.25
    fixed = _boundary(mesh)
    x0 = np.where(fixed[None, :], g, 0.0)
    x, iters, resid = _solve_el(mesh, lam, mu, rule, fixed, x0, None, "fp64", 1e-13)
    err = np.abs(x.cpu().numpy() - g).max() / np.abs(g).max()
    assert resid <= 1e-13 and iters > 0
    assert err <= 1e-10, err


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 3)])
@pytest.mark.parametrize("prec,rtol,tol", [("fp64", 1e-12, 1e-9), ("fp64_df", 1e-12, 1e-9), ("mixed", 1e-5, 1e-4)])
def test_elasticity_matches_dense_solve_of_oracle_operator(dim, n, prec, rtol, tol):
    mesh = _mesh(dim, n)
    rule = workloads.rule_for_dim(dim)
    rng = np.random.default_rng(dim + 30)
    E = rng.lognormal(0.0, 0.5, (rule.n_q, mesh.n_cells))
    nu = rng.uniform(0.2, 0.45, (rule.n_q, mesh.n_cells))
    lam, mu = workloads.cases.lame_from_young_poisson(E, nu)
    V = mesh.n_verts
    fixed = _boundary(mesh)
    g = np.stack([np.sin(mesh.coords[0] * 2.0), mesh.coords[1] - 0.5 * mesh.coords[0]] +
                 ([0.3 * mesh.coords[2]] if dim == 3 else []))
    b = np.where(fixed[None, :], 0.0, rng.uniform(-1, 1, (dim, V)) / V)
    if prec == "mixed":
        lam, mu = (a.astype(np.float32).astype(np.float64) for a in (lam, mu))
        b, g = (a.astype(np.float32).astype(np.float64) for a in (b, g))
    x0 = np.where(fixed[None, :], g, 0.0)
    x, iters, resid = _solve_el(mesh, lam, mu, rule, fixed, x0, b, prec, rtol)
    A = _oracle_elasticity_operator(mesh, lam, mu, rule)
    free = np.tile(~fixed, dim)
    fx = ~free
    ref = x0.ravel().copy()
    ref[free] = np.linalg.solve(A[np.ix_(free, free)], b.ravel()[free] - A[np.ix_(free, fx)] @ ref[fx])
    err = np.abs(x.cpu().numpy().astype(np.float64).ravel() - ref).max() / np.abs(ref).max()
    assert resid <= rtol
    assert err <= tol, (err, iters, resid)


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 3)])
@pytest.mark.parametrize("residual_prec", ["fp64", "fp64_df"])
def test_elasticity_refined_matches_dense_solve_of_oracle_operator(dim, n, residual_prec):
    """Mixed-precision refinement of the elasticity solve reaches the float64 solution of the
    oracle's assembled operator."""
    mesh = _mesh(dim, n)
    rule = workloads.rule_for_dim(dim)
    rng = np.random.default_rng(dim + 40)
    E = rng.lognormal(0.0, 0.5, (rule.n_q, mesh.n_cells))
    nu = rng.uniform(0.2, 0.45, (rule.n_q, mesh.n_cells))
    lam, mu = workloads.cases.lame_from_young_poisson(E, nu)
    V = mesh.n_verts
    fixed = _boundary(mesh)
    g = np.stack([mesh.coords[1] - 0.5 * mesh.coords[0]] + [np.cos(mesh.coords[0])] * (dim - 1))
    b = np.where(fixed[None, :], 0.0, rng.uniform(-1, 1, (dim, V)) / V)
    x0 = np.where(fixed[None, :], g, 0.0)
    coords, conn = to_dev(mesh.coords, torch.float64), to_dev(mesh.conn, torch.int32)
    ptr, idx = fem.fem_build_node2cell(conn, V)
    x = to_dev(x0, torch.float64)
    x, outer, inner, resid = fem.fem_pcg_elasticity_refined(
        coords, conn, to_dev(lam, torch.float64), to_dev(mu, torch.float64), rule.points, rule.weights, ptr, idx,
        to_dev(fixed.astype(np.uint8), torch.uint8), x, b=to_dev(b, torch.float64), max_outer=30, max_inner=20000,
        inner_rtol=1e-4, rtol=1e-12, residual_prec=residual_prec)
    A = _oracle_elasticity_operator(mesh, lam, mu, rule)
    free = np.tile(~fixed, dim)
    fx = ~free
    ref = x0.ravel().copy()
    ref[free] = np.linalg.solve(A[np.ix_(free, free)], b.ravel()[free] - A[np.ix_(free, fx)] @ ref[fx])
    err = np.abs(x.cpu().numpy().ravel() - ref).max() / np.abs(ref).max()
    assert resid <= 1e-12 and outer >= 2 and inner > 0
    assert err <= 1e-9, (err, outer, inner, resid)
