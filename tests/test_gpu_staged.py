"""Parity at the edges of the kernels' tilings, in every precision form.

Float64 inputs whose cell-indexed rows are 16-byte aligned (n_cells a multiple of 4) run
the persistent bulk-copy staged kernel: tiles of 1024 cells, a partial last tile, and
quadrature rules of any size (large rules whose stages do not fit shared memory take the
direct kernel); the float32 forms run the pair kernel on the same sizes. Also covered: the
bounded device-side wait and its error status.
"""

import numpy as np
import pytest
import torch

import oracle
import paper_1607_04245_gb300 as fem
import workloads
from gpu_util import PRECS, TOL, device_arrays, rel_err, residual

pytestmark = pytest.mark.gpu


def _cube_prefix(n_cells, seed=3):
    base = workloads.laplacian_cube_case(6 * 12 ** 3, seed=seed)  # 10,368 tets
    mesh = workloads.first_cells(base.mesh, n_cells)
    return workloads.Case("laplacian", mesh, base.rule, base.u[: mesh.n_verts], K=base.K[:, :n_cells].copy())


def _square_prefix(n_cells, seed=3):
    base = workloads.laplacian_square_case(80, seed=seed)  # 12,800 triangles
    mesh = workloads.first_cells(base.mesh, n_cells)
    return workloads.Case("laplacian", mesh, base.rule, base.u[: mesh.n_verts], K=base.K[:, :n_cells].copy())


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("n_cells", [4, 1020, 1024, 1028, 5 * 1024 + 8, 10 * 1024])
@pytest.mark.parametrize("prec", PRECS)
def test_tile_edges(dim, n_cells, prec):
    case = (_square_prefix if dim == 2 else _cube_prefix)(n_cells)
    c, d = device_arrays(case, prec)
    r = residual(c, d, prec)
    assert fem.fem_device_error() == 0
    assert rel_err(r, oracle.residual_for(c)) <= TOL[prec]


def _rule(dim, n_q, seed):
    """A positive-weight rule with n_q random points in the reference simplex (exactness
    does not matter for parity: both sides integrate with the same table)."""
    rng = np.random.default_rng(seed)
    lam = rng.dirichlet(np.ones(dim + 1), size=n_q)
    pts = np.ascontiguousarray(lam[:, 1:])
    w = rng.uniform(0.5, 1.5, n_q)
    w *= (1.0 / (2.0 if dim == 2 else 6.0)) / w.sum()
    return workloads.QuadRule(dim, pts, w)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("n_q", [1, 7, 32])
@pytest.mark.parametrize("prec", PRECS)
def test_quadrature_sizes(dim, n_q, prec):
    base = (_square_prefix if dim == 2 else _cube_prefix)(4096)
    rule = _rule(dim, n_q, seed=n_q)
    K = np.random.default_rng(11).lognormal(0.0, 1.0, (n_q, base.n_cells))
    case = workloads.Case("laplacian", base.mesh, rule, base.u, K=K)
    c, d = device_arrays(case, prec)
    r = residual(c, d, prec)
    assert rel_err(r, oracle.residual_for(c)) <= TOL[prec]


@pytest.mark.parametrize("n_cells", [4, 1028, 3 * 1024])
@pytest.mark.parametrize("prec", PRECS)
def test_adjoint_tile_edges(n_cells, prec):
    case = _cube_prefix(n_cells)
    case.adj = np.random.default_rng(5).uniform(-1.0, 1.0, (4, n_cells))
    c, d = device_arrays(case, prec)
    ptr, idx = fem.fem_build_node2cell(d["conn"], c.n_verts)
    dK, du = fem.fem_adjoint_laplacian(d["coords"], d["conn"], d["u"], d["K"], c.rule.points, c.rule.weights,
                                       d["adj"], ptr, idx, prec=prec)
    rK, ru = oracle.adjoint_for(c)
    assert rel_err(dK, rK) <= TOL[prec] and rel_err(du, ru) <= TOL[prec]


def test_bounded_wait_reports_timeout_and_context_survives():
    assert fem.fem_device_error() == 0
    fem.fem_selftest_wait(2_000_000)  # a 2 ms wait on a barrier phase nothing completes
    assert fem.fem_device_error() == -6  # FEM_ERR_TIMEOUT, then cleared
    assert fem.fem_device_error() == 0
    case = _cube_prefix(1024)
    c, d = device_arrays(case, "mixed")
    r = residual(c, d, "mixed")
    assert fem.fem_device_error() == 0
    assert rel_err(r, oracle.residual_for(c)) <= TOL["mixed"]
