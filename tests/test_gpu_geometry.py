"""Parity of the paper's precomputed-geometry layout (J^{-1} and det J per cell, Sec. 3
and the Appendix) with the CPU oracle, which computes the geometry from coordinates."""

import numpy as np
import pytest
import torch

import oracle
import paper_1607_04245_gb300 as fem
import workloads
from gpu_util import PRECS, TOL, device_arrays, rel_err

pytestmark = pytest.mark.gpu

# float32 geometry is rounded once per entry before the integration: on these meshes the
# element vectors then carry a relative error of a few float32 ulps
GEOM_TOL = {"fp64": 1e-12, "mixed": 2e-5, "fp32": 2e-5}


def _geom_residual(c, d, prec):
    geom = fem.fem_precompute_geometry(d["coords"], d["conn"], prec=prec)
    return fem.fem_integrate_laplacian_geom(d["conn"], c.n_verts, d["u"], d["K"], c.rule.points, c.rule.weights,
                                            geom, prec=prec), geom


@pytest.mark.parametrize("case_name", ["square8192", "cube1572864"])
@pytest.mark.parametrize("prec", PRECS)
def test_geometry_path_full(case_name, prec):
    case = workloads.laplacian_square_case() if case_name == "square8192" else workloads.laplacian_cube_case()
    c, d = device_arrays(case, prec)
    r, _ = _geom_residual(c, d, prec)
    assert rel_err(r, oracle.residual_for(c)) <= GEOM_TOL[prec]


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("n_cells", [1, 3, 4, 1027, 4100])
def test_geometry_path_ragged(dim, n_cells):
    base = workloads.laplacian_square_case(48) if dim == 2 else workloads.laplacian_cube_case(6 * 9 ** 3)
    mesh = workloads.first_cells(base.mesh, n_cells)
    case = workloads.Case("laplacian", mesh, base.rule, base.u[: mesh.n_verts], K=base.K[:, :n_cells].copy())
    for prec in PRECS:
        c, d = device_arrays(case, prec)
        r, _ = _geom_residual(c, d, prec)
        assert rel_err(r, oracle.residual_for(c)) <= GEOM_TOL[prec]


def test_geometry_values_invert_the_jacobian():
    """J^{-1} J = I and det J matches the product of the pivots, per cell (float64)."""
    case = workloads.laplacian_cube_case(6 * 5 ** 3)
    c, d = device_arrays(case, "fp64")
    geom = fem.fem_precompute_geometry(d["coords"], d["conn"], prec="fp64").cpu().numpy()
    x = c.mesh.coords[:, c.mesh.conn]  # (dim, NB, C)
    J = np.stack([x[:, j + 1, :] - x[:, 0, :] for j in range(3)], axis=1)  # J[i, j, c] = d x_i / d xi_j
    invJ = geom[:9].reshape(3, 3, -1)
    prod = np.einsum("ikc,kjc->ijc", invJ, J)
    assert np.abs(prod - np.eye(3)[:, :, None]).max() < 1e-12
    assert np.allclose(geom[9], np.linalg.det(np.moveaxis(J, 2, 0)), rtol=1e-12)
