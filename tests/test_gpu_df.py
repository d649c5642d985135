"""The float64-values, float32-pair-arithmetic form (FEM_FP64_DF) of the Laplacian residual
against the oracle at the float64 tolerance, including the fine 2048 x 1024 grid where the
Jacobian columns are 2^11 times smaller than the coordinates, inverted and skinny cells,
and ragged sizes."""

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


def test_df_is_laplacian_only():
    case = workloads.elasticity_case(2, 512)
    c, d = device_arrays(case, "fp64")
    with pytest.raises(fem.FemError):
        fem.fem_integrate_elasticity(d["coords"], d["conn"], d["u"], d["lam"], d["mu"], c.rule.points,
                                     c.rule.weights, prec="fp64_df")
