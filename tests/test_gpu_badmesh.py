"""The mesh-error status of the integrate entry points: a vertex id outside [0, n_verts)
(clamped in-kernel, so nothing is read out of bounds) or a cell with det J = 0 (a repeated
vertex, or vertices on one line/plane) sets a bit in the device error word, and the next
fem_device_error() returns FEM_ERR_BADMESH (-5) and clears it. Valid meshes leave it at 0,
and the cells of a mesh that are valid keep their results bit for bit."""

import numpy as np
import pytest
import torch

import paper_1607_04245_gb300 as fem
import workloads
from gpu_util import to_dev

pytestmark = pytest.mark.gpu

FEM_ERR_BADMESH = -5


def _lap_case(dim):
    return workloads.laplacian_square_case(12) if dim == 2 else workloads.laplacian_cube_case(6 * 5 ** 3)


def _flat_vertices(dim):
    """dim + 1 vertices on one line (2D) or plane (3D) whose Jacobian determinant is exactly 0."""
    if dim == 2:
        return np.array([[0.25, 0.5, 0.75], [0.5, 0.5, 0.5]])
    return np.array([[0.25, 0.75, 0.25, 0.75], [0.25, 0.25, 0.75, 0.75], [0.5, 0.5, 0.5, 0.5]])


def _broken(case, kind):
    """(coords, conn, u) of the case with cell 5 broken in the given way."""
    coords, conn, u = case.mesh.coords.copy(), case.mesh.conn.copy(), np.array(case.u, copy=True)
    V = case.n_verts
    if kind == "id_high":
        conn[0, 5] = V + 3
    elif kind == "id_negative":
        conn[1, 5] = -2
    elif kind == "repeated":
        conn[2, 5] = conn[1, 5]
    elif kind == "flat":
        flat = _flat_vertices(case.dim)
        coords = np.concatenate([coords, flat], axis=1)
        conn[:, 5] = np.arange(V, V + case.dim + 1)
        extra = np.zeros(u.shape[:-1] + (case.dim + 1,))
        u = np.concatenate([u, extra], axis=-1)
    return coords, conn, u


def _lap(coords, conn, u, K, rule, prec):
    dt = fem.value_dtype(prec)
    return fem.fem_integrate_laplacian(to_dev(coords, torch.float64), to_dev(conn, torch.int32), to_dev(u, dt),
                                       to_dev(K, dt), rule.points, rule.weights, prec=prec)


KINDS = ["id_high", "id_negative", "repeated", "flat"]


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32", "fp64_df"])
@pytest.mark.parametrize("kind", KINDS)
def test_laplacian_reports_bad_mesh(dim, prec, kind):
    case = _lap_case(dim)
    assert fem.fem_device_error() == 0
    good = _lap(case.mesh.coords, case.mesh.conn, case.u, case.K, case.rule, prec)
    assert fem.fem_device_error() == 0  # a valid mesh sets nothing
    coords, conn, u = _broken(case, kind)
    bad = _lap(coords, conn, u, case.K, case.rule, prec)
    assert fem.fem_device_error() == FEM_ERR_BADMESH
    assert fem.fem_device_error() == 0  # read and cleared
    keep = np.ones(case.n_cells, bool)
    keep[5] = False
    assert torch.equal(bad[:, keep], good[:, keep])


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp64_df"])
@pytest.mark.parametrize("kind", ["id_high", "repeated"])
def test_elasticity_reports_bad_mesh(dim, prec, kind):
    case = workloads.elasticity_case(dim, 2000 if dim == 2 else 3000)
    c = case if prec != "mixed" else case.rounded_to_f32()
    dt = fem.value_dtype(prec)
    coords, conn, u = _broken(c, kind)
    assert fem.fem_device_error() == 0
    fem.fem_integrate_elasticity(to_dev(coords, torch.float64), to_dev(conn, torch.int32), to_dev(u, dt),
                                 to_dev(c.lam, dt), to_dev(c.mu, dt), c.rule.points, c.rule.weights, prec=prec)
    assert fem.fem_device_error() == FEM_ERR_BADMESH
    assert fem.fem_device_error() == 0


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp64_df"])
def test_adjoint_reports_bad_mesh(prec):
    case = workloads.adjoint_case(6 * 5 ** 3)
    c = case if prec != "mixed" else case.rounded_to_f32()
    dt = fem.value_dtype(prec)
    coords, conn, u = _broken(c, "flat")
    d_conn = to_dev(conn, torch.int32)
    ptr, idx = fem.fem_build_node2cell(d_conn, coords.shape[1])
    assert fem.fem_device_error() == 0
    fem.fem_adjoint_laplacian(to_dev(coords, torch.float64), d_conn, to_dev(u, dt), to_dev(c.K, dt), c.rule.points,
                              c.rule.weights, to_dev(c.adj, dt), ptr, idx, prec=prec)
    assert fem.fem_device_error() == FEM_ERR_BADMESH
    assert fem.fem_device_error() == 0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["id_high", "flat"])
def test_reaction_geometry_fields_report_bad_mesh(prec, kind):
    case = _lap_case(3)
    c = case if prec == "fp64" else case.rounded_to_f32()
    dt = fem.value_dtype(prec)
    coords, conn, u = _broken(c, kind)
    V = coords.shape[1]
    d_coords, d_conn, d_u = to_dev(coords, torch.float64), to_dev(conn, torch.int32), to_dev(u, dt)
    a = to_dev(np.full(V, 1.5), dt)
    cq = to_dev(np.full((c.rule.n_q, c.n_cells), 0.7), dt)
    assert fem.fem_device_error() == 0
    fem.fem_integrate_reaction_diffusion(d_coords, d_conn, d_u, a, c.rule.points, c.rule.weights, c=cq, a_space=1,
                                         drift=0.5, prec=prec)
    assert fem.fem_device_error() == FEM_ERR_BADMESH
    geom = fem.fem_precompute_geometry(d_coords, d_conn, prec=prec)
    assert fem.fem_device_error() == FEM_ERR_BADMESH
    fem.fem_integrate_laplacian_geom(d_conn, V, d_u, to_dev(c.K, dt), c.rule.points, c.rule.weights, geom, prec=prec)
    assert fem.fem_device_error() == FEM_ERR_BADMESH  # a bad id, or the stored det J = 0
    fem.fem_integrate_laplacian_fields(d_coords, d_conn, torch.stack([d_u, d_u]), to_dev(c.K, dt), c.rule.points,
                                       c.rule.weights, prec=prec)
    assert fem.fem_device_error() == FEM_ERR_BADMESH
    assert fem.fem_device_error() == 0


def test_node2cell_and_closure_report_bad_ids():
    case = _lap_case(3)
    _, conn, u = _broken(case, "id_negative")
    d_conn = to_dev(conn, torch.int32)
    assert fem.fem_device_error() == 0
    fem.fem_build_node2cell(d_conn, case.n_verts)
    assert fem.fem_device_error() == FEM_ERR_BADMESH
    fem.fem_element_values(d_conn, case.n_verts, to_dev(u, torch.float64), prec="fp64")
    assert fem.fem_device_error() == FEM_ERR_BADMESH
    assert fem.fem_device_error() == 0
