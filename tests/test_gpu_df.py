"""The float64-values, float32-pair-arithmetic form (FEM_FP64_DF) of the Laplacian and
elasticity residuals against the oracle at the float64 tolerance, including the fine
2048 x 1024 grid where the Jacobian columns are 2^11 times smaller than the coordinates,
inverted and skinny cells, ragged sizes, and rigid motions."""

import numpy as np
import pytest
import torch

import oracle
import paper_1607_04245_gb300 as fem
import workloads
from gpu_util import device_arrays, rel_err, to_dev

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _res(case):
    c, d = device_arrays(case, "fp64")
    r = fem.fem_integrate_laplacian(d["coords"], d["conn"], d["u"], d["K"], c.rule.points, c.rule.weights,
                                    prec="fp64_df")
    return rel_err(r, oracle.residual_for(c))


def test_df_cube_full():
    assert _res(workloads.laplacian_cube_case()) <= TOL


def test_df_square_8192():
    assert _res(workloads.laplacian_square_case()) <= TOL


def test_df_fine_grid():
    mesh = workloads.square_mesh(2048, 1024, jitter=0.2, seed=4)
    rule = workloads.rule_for_dim(2)
    rng = np.random.default_rng(4)
    case = workloads.Case("laplacian", mesh, rule, rng.uniform(-1, 1, mesh.n_verts),
                          K=rng.lognormal(0, 1, (rule.n_q, mesh.n_cells)))
    assert _res(case) <= TOL


@pytest.mark.parametrize("dim", [2, 3])
def test_df_random_simplices(dim):
    rng = np.random.default_rng(dim)
    n = 5000
    X = rng.normal(size=(n, dim + 1, dim))
    X[: n // 10] *= np.array([1.0] * (dim - 1) + [1e-3])  # flattened (skinny) cells
    coords = X.reshape(-1, dim).T.copy() + 3.0  # away from the origin: cancellation in x_j - x_0
    conn = np.arange(n * (dim + 1), dtype=np.int32).reshape(n, dim + 1).T.copy()
    rule = workloads.rule_for_dim(dim)
    case = workloads.Case("laplacian", workloads.Mesh(dim, coords, conn), rule, rng.uniform(-1, 1, coords.shape[1]),
                          K=rng.lognormal(0, 1, (rule.n_q, n)))
    assert _res(case) <= TOL


@pytest.mark.parametrize("n_cells", [1, 3, 4097])
def test_df_ragged(n_cells):
    base = workloads.laplacian_cube_case(6 * 9 ** 3)
    mesh = workloads.first_cells(base.mesh, n_cells)
    case = workloads.Case("laplacian", mesh, base.rule, base.u[: mesh.n_verts], K=base.K[:, :n_cells].copy())
    assert _res(case) <= TOL


def test_df_refused_where_not_offered():
    """The reaction-diffusion entry has no double-float form: an argument error."""
    case = workloads.laplacian_square_case(8)
    c, d = device_arrays(case, "fp64")
    a = torch.ones(c.n_verts, dtype=torch.float64, device="cuda")
    with pytest.raises(fem.FemError):
        fem.fem_integrate_reaction_diffusion(d["coords"], d["conn"], d["u"], a, c.rule.points, c.rule.weights,
                                             prec="fp64_df")


# ---- linear elasticity in the double-float form


def _el_res(case):
    c, d = device_arrays(case, "fp64")
    r = fem.fem_integrate_elasticity(d["coords"], d["conn"], d["u"], d["lam"], d["mu"], c.rule.points,
                                     c.rule.weights, prec="fp64_df")
    return r, rel_err(r, oracle.residual_for(c))


@pytest.mark.parametrize("dim", [2, 3])
def test_df_elasticity_full_size(dim):
    """2^22 triangles / 2^21 tets, per-point Lame coefficients, against the oracle."""
    r, err = _el_res(workloads.elasticity_case(dim))
    assert err <= TOL, err


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("n_cells", [1, 3, 5, 1027])
def test_df_elasticity_ragged(dim, n_cells):
    base = workloads.elasticity_case(dim, 2 * 32 * 32 if dim == 2 else 6 * 12 ** 3)
    mesh = workloads.first_cells(base.mesh, n_cells)
    case = workloads.Case("elasticity", mesh, base.rule, base.u[:, : mesh.n_verts].copy(),
                          lam=base.lam[:, :n_cells].copy(), mu=base.mu[:, :n_cells].copy())
    assert _el_res(case)[1] <= TOL


@pytest.mark.parametrize("dim", [2, 3])
def test_df_elasticity_rigid_motions_and_sums(dim):
    """Rigid motions give zero element vectors; every component's entries sum to zero."""
    case = workloads.elasticity_case(dim, 2 * 32 * 32 if dim == 2 else 6 * 12 ** 3)
    x = case.mesh.coords
    if dim == 2:
        U = np.stack([0.3 - 0.7 * x[1], -1.1 + 0.7 * x[0]])
    else:
        w = np.array([0.2, -0.5, 0.9])
        U = np.array([0.1, 0.2, -0.3])[:, None] + np.cross(w, x.T).T
    rigid = workloads.Case("elasticity", case.mesh, case.rule, U, lam=case.lam, mu=case.mu)
    r, _ = _el_res(rigid)
    # scale: the element vectors of a pure stretch of the same magnitude (u = x)
    stretch = workloads.Case("elasticity", case.mesh, case.rule, x.copy(), lam=case.lam, mu=case.mu)
    scale = np.abs(oracle.residual_for(stretch)).max()
    assert r.abs().max().item() <= TOL * scale
    r2, _ = _el_res(case)
    sums = r2.view(dim + 1, dim, -1).sum(0).abs().max().item()
    assert sums <= 1e-14 * r2.abs().max().item()


# ---- the adjoint in the double-float form


def _adj(case, prec):
    c, d = device_arrays(case, "fp64")
    q = c.rule
    ptr, idx = fem.fem_build_node2cell(d["conn"], c.n_verts)
    dK, du = fem.fem_adjoint_laplacian(d["coords"], d["conn"], d["u"], d["K"], q.points, q.weights, d["adj"], ptr,
                                       idx, prec=prec)
    return c, dK, du


def test_df_adjoint_full_size():
    """dJ/dK and dJ/du on the 1,572,864-tet workload against the oracle at the float64
    tolerance, and against the float64 form."""
    case = workloads.adjoint_case()
    c, dK, du = _adj(case, "fp64_df")
    rK, ru = oracle.adjoint_for(c)
    assert rel_err(dK, rK) <= TOL and rel_err(du, ru) <= TOL
    _, dK64, du64 = _adj(case, "fp64")
    assert rel_err(dK, dK64.double().cpu().numpy()) <= TOL and rel_err(du, du64.double().cpu().numpy()) <= TOL


@pytest.mark.parametrize("n_cells", [1, 5, 1027])
def test_df_adjoint_ragged_and_reproducible(n_cells):
    base = workloads.adjoint_case(6 * 12 ** 3)
    mesh = workloads.first_cells(base.mesh, n_cells)
    case = workloads.Case("laplacian", mesh, base.rule, base.u[: mesh.n_verts], K=base.K[:, :n_cells].copy(),
                          adj=base.adj[:, :n_cells].copy())
    c, dK, du = _adj(case, "fp64_df")
    rK, ru = oracle.adjoint_for(c)
    assert rel_err(dK, rK) <= TOL and rel_err(du, ru) <= TOL
    _, dK2, du2 = _adj(case, "fp64_df")
    assert torch.equal(dK, dK2) and torch.equal(du, du2)
