"""Parity of the CUDA elasticity residual (fem_integrate_elasticity) with the CPU oracle."""

import numpy as np
import pytest
import torch

import oracle
import paper_1607_04245_gb300 as fem
import workloads
from gpu_util import PRECS, TOL, as_input, device_arrays, rel_err, residual, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[2, 3])
def elast(request):
    return workloads.elasticity_case(request.param)  # 2^22 triangles / 2^21 tets


@pytest.mark.parametrize("prec", PRECS)
def test_full_size(elast, prec):
    c, d = device_arrays(elast, prec)
    r = residual(c, d, prec)
    torch.cuda.synchronize()
    err = rel_err(r, oracle.residual_for(c))
    print(f"{elast.name} {prec}: rel max-norm err {err:.3e}")
    assert err <= TOL[prec]
    if prec == "mixed":
        err64 = rel_err(r, oracle.residual_for(elast))  # the unrounded float64 u, lambda, mu
        print(f"{elast.name} mixed vs the float64 inputs: {err64:.3e}")
        assert err64 <= TOL["mixed"]
    # per-component element sums vanish
    dim = elast.dim
    s = r.double().view(dim + 1, dim, -1).sum(0).abs().max().item()
    assert s <= (1e-15 if prec == "fp64" else 1e-6) * r.double().abs().max().item()


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("n_cells", [1, 3, 6, 1029, 6 * 5 ** 3 - 1])
@pytest.mark.parametrize("prec", PRECS)
def test_ragged_sizes(dim, n_cells, prec):
    case = workloads.elasticity_case(dim, n_cells)
    c, d = device_arrays(case, prec)
    r = residual(c, d, prec)
    torch.cuda.synchronize()
    assert rel_err(r, oracle.residual_for(c)) <= TOL[prec]


@pytest.mark.parametrize("dim", [2, 3])
def test_rigid_motions(dim):
    case = workloads.elasticity_case(dim, 2 * 32 * 32 if dim == 2 else 6 * 12 ** 3)
    x = case.mesh.coords
    if dim == 2:
        u = np.array([[0.1], [-0.2]]) + 0.3 * np.stack([-x[1], x[0]])
    else:
        u = np.array([[0.1], [-0.2], [0.05]]) + np.cross(np.array([0.3, -0.1, 0.2]), x.T).T
    for prec in ("fp64", "mixed"):
        c, d = device_arrays(case, prec)
        d["u"] = to_dev(u, fem.value_dtype(prec))
        r = residual(c, d, prec)
        torch.cuda.synchronize()
        scale = np.abs(oracle.elasticity(x, case.mesh.conn, 100 * case.u, c.lam, c.mu, case.rule.points,
                                         case.rule.weights)).max()
        assert r.double().abs().max().item() <= (1e-13 if prec == "fp64" else 1e-5) * scale


def test_paper_listing_special_case():
    """lambda = 0, mu = 1/2: the symmetric-gradient pointwise function of Sec. 6."""
    case = workloads.elasticity_case(2, 2 * 40 * 40)
    case.lam = np.zeros_like(case.lam)
    case.mu = np.full_like(case.mu, 0.5)
    c, d = device_arrays(case, "fp64")
    r = residual(c, d, "fp64")
    torch.cuda.synchronize()
    assert rel_err(r, oracle.residual_for(c)) <= TOL["fp64"]
