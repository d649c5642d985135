"""The assembly sum E^T of Eq. 2 (fem_gather_nodes) for the Laplacian (one component per
vertex) and for elasticity (dim components per vertex), in every precision form: the
nodal sums of the kernels' own element vectors against the same sums formed on the host,
and against the assembly of the CPU oracle's element vectors; repeated calls are bitwise
identical (fixed summation order, no atomics)."""

import numpy as np
import pytest
import torch

import oracle
import paper_1607_04245_gb300 as fem
import workloads
from gpu_util import TOL, rel_err, residual, to_dev

pytestmark = pytest.mark.gpu

TOL_ASM = dict(TOL, fp64_df=1e-12)
PRECS = ("fp64", "mixed", "fp32", "fp64_df")


def _case(physics, dim, n_cells):
    if physics == "laplacian":
        if dim == 3:
            return workloads.laplacian_cube_case(n_cells)
        return workloads.laplacian_square_case(n_cells)  # n x n squares, 2 n^2 triangles
    return workloads.elasticity_case(dim, n_cells)


def _device(case, prec):
    c = case if prec in ("fp64", "fp64_df") else case.rounded_to_f32()
    dt = fem.value_dtype(prec)
    d = {"coords": to_dev(c.mesh.coords, torch.float64), "conn": to_dev(c.mesh.conn, torch.int32),
         "u": to_dev(c.u, dt)}
    for name in ("K", "lam", "mu"):
        if getattr(c, name) is not None:
            d[name] = to_dev(getattr(c, name), dt)
    return c, d


def _assemble_host(elem, conn, n_comp, V):
    """E^T on the host: out[k][n] = sum over (e, a) with conn[a][e] = n of elem[a*n_comp + k][e]."""
    out = np.zeros((n_comp, V))
    for a in range(conn.shape[0]):
        for k in range(n_comp):
            np.add.at(out[k], conn[a], elem[a * n_comp + k])
    return out


CASES = [("laplacian", 2, 37), ("laplacian", 3, 4097), ("laplacian", 3, 24576),
         ("elasticity", 2, 2738), ("elasticity", 2, 20000), ("elasticity", 3, 4097), ("elasticity", 3, 24576)]


@pytest.mark.parametrize("physics,dim,size", CASES)
@pytest.mark.parametrize("prec", PRECS)
def test_gather_nodes_assembles_element_vectors(physics, dim, size, prec):
    case = _case(physics, dim, size)
    c, d = _device(case, prec)
    V, C = c.n_verts, c.n_cells
    n_comp = c.n_comp
    elem = residual(c, d, prec)
    ptr, idx = fem.fem_build_node2cell(d["conn"], V)
    nodal = fem.fem_gather_nodes(elem, ptr, idx, V, dim, prec=prec)
    torch.cuda.synchronize()
    assert nodal.shape == (n_comp, V) and nodal.dtype == fem.value_dtype(prec)
    # the kernel's own element vectors summed on the host: only the summation order differs
    host = _assemble_host(elem.double().cpu().numpy(), c.mesh.conn, n_comp, V)
    f64 = prec in ("fp64", "fp64_df")
    assert rel_err(nodal, host) <= (1e-13 if f64 else 2e-7)
    # against the assembled oracle element vectors
    ref = _assemble_host(oracle.residual_for(c), c.mesh.conn, n_comp, V)
    assert rel_err(nodal, ref) <= TOL_ASM[prec]
    # fixed order: a second call and a call into a caller-owned output are bitwise identical
    again = torch.full_like(nodal, float("nan"))
    fem.fem_gather_nodes(elem, ptr, idx, V, dim, out=again, prec=prec)
    torch.cuda.synchronize()
    assert torch.equal(nodal, again)


@pytest.mark.parametrize("dim", [2, 3])
def test_gather_nodes_rigid_motion_and_interior_zero(dim):
    """Assembled elasticity residual of a rigid motion vanishes at every vertex; for a linear
    displacement with constant Lame parameters it vanishes at interior vertices (patch test)."""
    case = workloads.elasticity_case(dim, 2 * 32 ** 2 if dim == 2 else 6 * 8 ** 3)  # whole meshes
    m = case.mesh
    V = m.n_verts
    x = m.coords
    lam = np.full_like(case.lam, 1.3)
    mu = np.full_like(case.mu, 0.7)
    if dim == 2:
        u_rigid = np.stack([0.3 - 0.2 * x[1], -0.1 + 0.2 * x[0]])
    else:
        w = np.array([0.2, -0.1, 0.05])
        u_rigid = np.array([0.3, -0.1, 0.2])[:, None] + np.cross(w, x.T).T
    A = np.arange(1, dim * dim + 1, dtype=np.float64).reshape(dim, dim) / 10.0
    u_lin = A @ x + 0.25
    coords, conn = to_dev(x, torch.float64), to_dev(m.conn, torch.int32)
    ptr, idx = fem.fem_build_node2cell(conn, V)
    boundary = np.any((np.abs(x) < 1e-14) | (np.abs(x - 1.0) < 1e-14), axis=0)
    lam_d, mu_d = to_dev(lam, torch.float64), to_dev(mu, torch.float64)
    res = lambda u: fem.fem_integrate_elasticity(coords, conn, to_dev(u, torch.float64), lam_d, mu_d,
                                                 case.rule.points, case.rule.weights, prec="fp64")
    # rounding only: against the element vectors of a field with gradients of the same size
    scale = np.abs(res(u_lin).cpu().numpy()).max()
    for u, mask in ((u_rigid, np.ones(V, bool)), (u_lin, ~boundary)):
        nodal = fem.fem_gather_nodes(res(u), ptr, idx, V, dim, prec="fp64").cpu().numpy()
        assert np.abs(nodal[:, mask]).max() <= 1e-12 * scale


def test_gather_nodes_argument_errors():
    conn = torch.zeros((4, 8), dtype=torch.int32, device="cuda")
    ptr, idx = fem.fem_build_node2cell(conn, 5)
    elem = torch.zeros((4, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        fem.fem_gather_nodes(elem[:3], ptr, idx, 5, 3, prec="fp64")  # rows not a multiple of dim+1
    with pytest.raises(ValueError):
        fem.fem_gather_nodes(elem, ptr, idx, 5, 3, prec="mixed")  # float64 elem for a float32 form
    out = fem.fem_gather_nodes(torch.zeros((0, 0), dtype=torch.float32, device="cuda").reshape(4, 0),
                               fem.fem_build_node2cell(torch.zeros((4, 0), dtype=torch.int32, device="cuda"), 3)[0],
                               torch.zeros(0, dtype=torch.int32, device="cuda"), 3, 3, prec="mixed")
    torch.cuda.synchronize()
    assert out.shape == (1, 3) and torch.all(out == 0)
