"""Parity of the several-fields Laplacian residual (fem_integrate_laplacian_fields) with
the CPU oracle, field by field, and with the single-field entry: bitwise in float64 and
against the single-field per-cell path (misaligned rows) in the float32 forms."""

import numpy as np
import pytest
import torch

import oracle
import paper_1607_04245_gb300 as fem
import workloads
from gpu_util import PRECS, TOL, as_input, misaligned, rel_err, to_dev

pytestmark = pytest.mark.gpu


def _fields(case, n_fields, seed=0):
    rng = np.random.default_rng(seed + 17)
    return rng.uniform(-1.0, 1.0, (n_fields, case.n_verts))


def _device(case, U, prec):
    c = as_input(case, prec)
    dt = fem.value_dtype(prec)
    U = U if prec == "fp64" else U.astype(np.float32).astype(np.float64)
    return c, U, {"coords": to_dev(c.mesh.coords, torch.float64), "conn": to_dev(c.mesh.conn, torch.int32),
                  "U": to_dev(U, dt), "K": to_dev(c.K, dt)}


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("n_fields", [1, 3, 8])
@pytest.mark.parametrize("prec", PRECS)
def test_fields_match_oracle(dim, n_fields, prec):
    case = workloads.laplacian_square_case() if dim == 2 else workloads.laplacian_cube_case(6 * 24 ** 3)
    c, U, d = _device(case, _fields(case, n_fields), prec)
    q = c.rule
    r = fem.fem_integrate_laplacian_fields(d["coords"], d["conn"], d["U"], d["K"], q.points, q.weights, prec=prec)
    assert r.shape == (n_fields, dim + 1, c.n_cells)
    for f in range(n_fields):
        ref = oracle.laplacian(c.mesh.coords, c.mesh.conn, U[f], c.K, q.points, q.weights)
        assert rel_err(r[f], ref) <= TOL[prec], f


@pytest.mark.parametrize("prec", PRECS)
def test_fields_equal_single_field_per_cell_path(prec):
    """Misaligned rows send the single-field call to its per-cell kernel, whose arithmetic
    the several-fields kernel repeats per field (float64: also the staged kernel's)."""
    case = workloads.laplacian_cube_case(6 * 16 ** 3)
    c, U, d = _device(case, _fields(case, 4, seed=1), prec)
    q = c.rule
    r = fem.fem_integrate_laplacian_fields(d["coords"], d["conn"], d["U"], d["K"], q.points, q.weights, prec=prec)
    conn_m, K_m = misaligned(d["conn"]), misaligned(d["K"])
    for f in range(4):
        one = fem.fem_integrate_laplacian(d["coords"], conn_m, misaligned(d["U"][f].contiguous()), K_m, q.points,
                                          q.weights, out=misaligned(torch.empty_like(r[f])), prec=prec)
        assert torch.equal(r[f], one), f
        if prec == "fp64":
            aligned = fem.fem_integrate_laplacian(d["coords"], d["conn"], d["U"][f].contiguous(), d["K"], q.points,
                                                  q.weights, prec=prec)
            assert torch.equal(r[f], aligned), f


@pytest.mark.parametrize("n_cells", [1, 2, 3, 5, 1027, 4096])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fields_ragged(n_cells, prec):
    base = workloads.laplacian_cube_case(6 * 16 ** 3)
    mesh = workloads.first_cells(base.mesh, n_cells)
    case = workloads.Case("laplacian", mesh, base.rule, base.u[: mesh.n_verts], K=base.K[:, :n_cells].copy())
    c, U, d = _device(case, _fields(case, 5, seed=2), prec)
    q = c.rule
    r = fem.fem_integrate_laplacian_fields(d["coords"], d["conn"], d["U"], d["K"], q.points, q.weights, prec=prec)
    for f in range(5):
        ref = oracle.laplacian(c.mesh.coords, c.mesh.conn, U[f], c.K, q.points, q.weights)
        assert rel_err(r[f], ref) <= TOL[prec], f


def test_fields_mixed_fallback_on_slivers():
    """Flattened cells fail the mixed form's shape test and are recomputed in float64 for
    every field."""
    rng = np.random.default_rng(9)
    n = 4000
    X = rng.normal(size=(n, 4, 3))
    X[: n // 4, :, 2] *= 1e-4  # nearly flat tetrahedra
    coords = X.reshape(-1, 3).T.copy() + 2.0
    conn = np.arange(4 * n, dtype=np.int32).reshape(n, 4).T.copy()
    rule = workloads.rule_for_dim(3)
    case = workloads.Case("laplacian", workloads.Mesh(3, coords, conn), rule, np.zeros(coords.shape[1]),
                          K=rng.lognormal(0, 1, (rule.n_q, n)))
    c, U, d = _device(case, _fields(case, 3, seed=3), "mixed")
    r = fem.fem_integrate_laplacian_fields(d["coords"], d["conn"], d["U"], d["K"], rule.points, rule.weights,
                                           prec="mixed")
    for f in range(3):
        ref = oracle.laplacian(c.mesh.coords, c.mesh.conn, U[f], c.K, rule.points, rule.weights)
        assert rel_err(r[f], ref) <= TOL["mixed"], f


def test_zero_fields_is_a_noop_and_bad_count_is_refused():
    case = workloads.laplacian_square_case(8)
    c, U, d = _device(case, _fields(case, 1), "fp64")
    q = c.rule
    empty = torch.empty((0, c.n_verts), dtype=torch.float64, device="cuda")
    r = fem.fem_integrate_laplacian_fields(d["coords"], d["conn"], empty, d["K"], q.points, q.weights, prec="fp64")
    assert r.shape == (0, 3, c.n_cells)
    with pytest.raises(fem.FemError):
        fem.fem_integrate_laplacian_fields(d["coords"], d["conn"], d["U"], d["K"], q.points, q.weights,
                                           prec="fp64_df")
