"""Parity of the reaction-diffusion kernel (Eq. 2 with f0 = c u + g grad a . grad u and
f1 = a grad u; Eq. 8 with the auxiliary field a in P1 or P0) with the CPU oracle, on the
workloads' meshes with the paper's benchmark coefficient form (a P1 field), a per-point
reaction and the first-order term along grad a."""

import numpy as np
import pytest
import torch

import oracle
import paper_1607_04245_gb300 as fem
import workloads
from gpu_util import PRECS, TOL, misaligned, rel_err, to_dev

pytestmark = pytest.mark.gpu


def _case(dim, n_cells=None, seed=0):
    if dim == 2:
        base = workloads.laplacian_square_case(64, seed=seed)
    else:
        base = workloads.laplacian_cube_case(n_cells or 6 * 32 ** 3, seed=seed)
    rng = np.random.default_rng(seed + 100)
    C, V = base.n_cells, base.n_verts
    a_p1 = rng.lognormal(0.0, 0.5, V)
    a_p0 = rng.lognormal(0.0, 0.5, C)
    c = rng.uniform(0.5, 2.0, (base.rule.n_q, C))
    return base, a_p1, a_p0, c


def _gpu(base, a, a_space, c, prec, drift=0.0):
    dt = fem.value_dtype(prec)
    m, q = base.mesh, base.rule
    return fem.fem_integrate_reaction_diffusion(to_dev(m.coords, torch.float64), to_dev(m.conn, torch.int32),
                                                to_dev(base.u, dt), to_dev(a, dt), q.points, q.weights,
                                                c=None if c is None else to_dev(c, dt), a_space=a_space,
                                                drift=drift, prec=prec)


def _run(base, a, a_space, c, prec, drift=0.0):
    cast = (lambda x: x) if prec == "fp64" else (lambda x: np.asarray(x, dtype=np.float32).astype(np.float64))
    u, a, c = cast(base.u), cast(a), None if c is None else cast(c)
    m, q = base.mesh, base.rule
    r = _gpu(base, a, a_space, c, prec, drift)
    ref = oracle.reaction_diffusion(m.coords, m.conn, u, a, a_space, c, q.points, q.weights, drift=drift)
    return rel_err(r, ref)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("a_space", [0, 1])
@pytest.mark.parametrize("react", [False, True])
@pytest.mark.parametrize("drift", [0.0, 1.3])
@pytest.mark.parametrize("prec", PRECS)
def test_reaction_diffusion_parity(dim, a_space, react, drift, prec):
    base, a_p1, a_p0, c = _case(dim)
    err = _run(base, a_p1 if a_space == 1 else a_p0, a_space, c if react else None, prec, drift)
    assert err <= TOL[prec], err


@pytest.mark.parametrize("n_cells", [1, 2, 3, 5, 1027])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_reaction_diffusion_ragged_with_drift(n_cells, prec):
    base, a_p1, _, c = _case(3)
    mesh = workloads.first_cells(base.mesh, n_cells)
    case = workloads.Case("laplacian", mesh, base.rule, base.u[: mesh.n_verts], K=base.K[:, :n_cells].copy())
    assert _run(case, a_p1[: mesh.n_verts], 1, c[:, :n_cells].copy(), prec, drift=-0.7) <= TOL[prec]


@pytest.mark.parametrize("n_cells", [4, 1020, 1024, 1028, 3076])
@pytest.mark.parametrize("a_space", [0, 1])
@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_vector_rows_match_oracle_and_per_cell_path(n_cells, a_space, prec):
    """Aligned rows and a cell count divisible by 4 take the four-cells-per-thread kernel with
    16-byte row accesses; misaligned rows take the one-cell-per-thread kernel, whose per-cell
    arithmetic is the same: the two agree bitwise."""
    base, a_p1, a_p0, c = _case(3)
    mesh = workloads.first_cells(base.mesh, n_cells)
    a = (a_p1[: mesh.n_verts] if a_space == 1 else a_p0[:n_cells]).copy()
    case = workloads.Case("laplacian", mesh, base.rule, base.u[: mesh.n_verts], K=base.K[:, :n_cells].copy())
    cc = c[:, :n_cells].copy()
    drift = 0.6 if a_space == 1 else 0.0
    assert _run(case, a, a_space, cc, prec, drift) <= TOL[prec]
    dt = fem.value_dtype(prec)
    m, q = case.mesh, case.rule
    coords, conn = to_dev(m.coords, torch.float64), to_dev(m.conn, torch.int32)
    u, ad, cd = to_dev(case.u, dt), to_dev(a, dt), to_dev(cc, dt)
    staged = fem.fem_integrate_reaction_diffusion(coords, conn, u, ad, q.points, q.weights, c=cd, a_space=a_space,
                                                  drift=drift, prec=prec)
    per_cell = fem.fem_integrate_reaction_diffusion(coords, misaligned(conn), u, ad, q.points, q.weights,
                                                    c=misaligned(cd), a_space=a_space, drift=drift, prec=prec)
    assert torch.equal(staged, per_cell)


def test_drift_ignored_for_p0_coefficient():
    """grad a = 0 inside a cell for a P0 field: the result is bitwise the one without drift."""
    base, _, a_p0, c = _case(3)
    assert torch.equal(_gpu(base, a_p0, 0, c, "mixed", 2.5), _gpu(base, a_p0, 0, c, "mixed", 0.0))


def test_reaction_diffusion_full_size_mixed():
    base, a_p1, _, c = _case(3, n_cells=1572864)
    assert _run(base, a_p1, 1, c, "mixed") <= TOL["mixed"]
    assert _run(base, a_p1, 1, c, "mixed", drift=0.9) <= TOL["mixed"]


def test_requires_quadrature_points():
    base, a_p1, _, _ = _case(2)
    m = base.mesh
    with pytest.raises(ValueError):
        fem.fem_integrate_reaction_diffusion(to_dev(m.coords, torch.float64), to_dev(m.conn, torch.int32),
                                             to_dev(base.u, torch.float64), to_dev(a_p1, torch.float64), None,
                                             base.rule.weights, prec="fp64")
