"""Parity of the paper's thread-transposition kernel (Sec. 3, rebuilt as an ablation) with
the CPU oracle, over its two batch parameters (cells per batch, batches per block)."""

import numpy as np
import pytest
import torch

import oracle
import paper_1607_04245_gb300 as fem
import workloads
from gpu_util import device_arrays, rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}


def _run(case, prec, cpb, bpb):
    c, d = device_arrays(case, prec)
    geom = fem.fem_precompute_geometry(d["coords"], d["conn"], prec=prec)
    ue = fem.fem_element_values(d["conn"], c.n_verts, d["u"], prec=prec)
    r = fem.fem_integrate_laplacian_transposed(ue, d["K"], c.rule.points, c.rule.weights, geom, cells_per_batch=cpb,
                                               batches_per_block=bpb, prec=prec)
    return rel_err(r, oracle.residual_for(c))


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("cpb,bpb", [(32, 1), (64, 4), (128, 3)])
def test_transposed_parity(dim, prec, cpb, bpb):
    case = workloads.laplacian_square_case(64) if dim == 2 else workloads.laplacian_cube_case(6 * 20 ** 3)
    assert _run(case, prec, cpb, bpb) <= TOL[prec]


@pytest.mark.parametrize("n_cells", [1, 31, 33, 1000, 4097])
def test_transposed_ragged(n_cells):
    base = workloads.laplacian_cube_case(6 * 9 ** 3)
    mesh = workloads.first_cells(base.mesh, n_cells)
    case = workloads.Case("laplacian", mesh, base.rule, base.u[: mesh.n_verts], K=base.K[:, :n_cells].copy())
    assert _run(case, "fp32", 256, 2) <= TOL["fp32"]
    assert _run(case, "fp64", 64, 5) <= TOL["fp64"]


def test_transposed_full_size():
    assert _run(workloads.laplacian_cube_case(), "fp32", 128, 4) <= TOL["fp32"]


def test_transposed_rejects_bad_parameters():
    case = workloads.laplacian_cube_case(6 * 4 ** 3)
    c, d = device_arrays(case, "fp64")
    geom = fem.fem_precompute_geometry(d["coords"], d["conn"], prec="fp64")
    ue = fem.fem_element_values(d["conn"], c.n_verts, d["u"], prec="fp64")
    for cpb, bpb in ((48, 1), (256, 1), (64, 0)):
        with pytest.raises(fem.FemError):
            fem.fem_integrate_laplacian_transposed(ue, d["K"], c.rule.points, c.rule.weights, geom,
                                                   cells_per_batch=cpb, batches_per_block=bpb, prec="fp64")
