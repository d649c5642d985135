"""Parity of the reaction-diffusion kernel (Eq. 2 with f0 = c u and f1 = a grad u; Eq. 8
with the auxiliary field a in P1 or P0) with the CPU oracle, on the workloads' meshes
with the paper's benchmark coefficient form (a P1 field) and a per-point reaction."""

import numpy as np
import pytest
import torch

import oracle
import paper_1607_04245_gb300 as fem
import workloads
from gpu_util import PRECS, TOL, rel_err, to_dev

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


def _run(base, a, a_space, c, prec):
    dt = fem.value_dtype(prec)
    cast = (lambda x: x) if prec == "fp64" else (lambda x: np.asarray(x, dtype=np.float32).astype(np.float64))
    u, a, c = cast(base.u), cast(a), None if c is None else cast(c)
    m, q = base.mesh, base.rule
    r = fem.fem_integrate_reaction_diffusion(to_dev(m.coords, torch.float64), to_dev(m.conn, torch.int32),
                                             to_dev(u, dt), to_dev(a, dt), q.points, q.weights,
                                             c=None if c is None else to_dev(c, dt), a_space=a_space, prec=prec)
    ref = oracle.reaction_diffusion(m.coords, m.conn, u, a, a_space, c, q.points, q.weights)
    return rel_err(r, ref)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("a_space", [0, 1])
@pytest.mark.parametrize("react", [False, True])
@pytest.mark.parametrize("prec", PRECS)
def test_reaction_diffusion_parity(dim, a_space, react, prec):
    base, a_p1, a_p0, c = _case(dim)
    err = _run(base, a_p1 if a_space == 1 else a_p0, a_space, c if react else None, prec)
    assert err <= TOL[prec], err


def test_reaction_diffusion_full_size_mixed():
    base, a_p1, _, c = _case(3, n_cells=1572864)
    assert _run(base, a_p1, 1, c, "mixed") <= TOL["mixed"]


def test_requires_quadrature_points():
    base, a_p1, _, _ = _case(2)
    m = base.mesh
    with pytest.raises(ValueError):
        fem.fem_integrate_reaction_diffusion(to_dev(m.coords, torch.float64), to_dev(m.conn, torch.int32),
                                             to_dev(base.u, torch.float64), to_dev(a_p1, torch.float64), None,
                                             base.rule.weights, prec="fp64")
