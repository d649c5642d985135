"""The prepared vertex records (fem_prepare_vertices, fem_integrate_laplacian_prepared): the
mixed-form Laplacian from per-mesh (hi, lo) coordinate records gives bitwise the element
vectors of fem_integrate_laplacian, at full and ragged (even) sizes, with its float64
recomputation of badly shaped cells and its mesh check."""

import numpy as np
import pytest
import torch

import oracle
import paper_1607_04245_gb300 as fem
import workloads
from gpu_util import TOL, device_arrays, rel_err, residual

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,n", [(3, 1572864), (3, 6 * 7 ** 3 - 2), (2, 8192), (2, 2 * 37 ** 2)])
def test_prepared_equals_the_integrate_entry(dim, n):
    case = workloads.laplacian_cube_case(n) if dim == 3 else workloads.laplacian_square_case(int(round((n / 2) ** 0.5)))
    c, d = device_arrays(case, "mixed")
    rec = fem.fem_prepare_vertices(d["coords"])
    r = fem.fem_integrate_laplacian_prepared(d["coords"], rec, d["conn"], d["u"], d["K"], c.rule.points, c.rule.weights)
    ref = residual(c, d, "mixed")
    torch.cuda.synchronize()
    assert torch.equal(r, ref)
    assert rel_err(r, oracle.residual_for(c)) <= TOL["mixed"]


def test_prepared_fallback_and_mesh_check():
    case = workloads.laplacian_cube_case(6 * 5 ** 3)
    c, d = device_arrays(case, "mixed")
    old = fem.fem_get_mixed_threshold()
    try:
        fem.fem_set_mixed_threshold(2.0)  # every cell recomputed in float64
        rec = fem.fem_prepare_vertices(d["coords"])
        r = fem.fem_integrate_laplacian_prepared(d["coords"], rec, d["conn"], d["u"], d["K"], c.rule.points,
                                                 c.rule.weights)
        assert torch.equal(r, residual(c, d, "mixed"))
    finally:
        fem.fem_set_mixed_threshold(old)
    assert fem.fem_device_error() == 0
    bad = d["conn"].clone()
    bad[1, 4] = c.n_verts + 2
    fem.fem_integrate_laplacian_prepared(d["coords"], rec, bad, d["u"], d["K"], c.rule.points, c.rule.weights)
    assert fem.fem_device_error() == -5


def test_prepared_argument_errors():
    case = workloads.laplacian_cube_case(6 * 3 ** 3)
    c, d = device_arrays(case, "mixed")
    rec = fem.fem_prepare_vertices(d["coords"])
    with pytest.raises(fem.FemError):  # an odd cell count
        fem.fem_integrate_laplacian_prepared(d["coords"], rec, d["conn"][:, :5].contiguous(), d["u"],
                                             d["K"][:, :5].contiguous(), c.rule.points, c.rule.weights)
