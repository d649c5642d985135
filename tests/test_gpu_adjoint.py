"""The adjoint of the Laplacian residual on the GPU: vertex-to-cell lists, parity of
dJ/dK and dJ/du with the oracle, central differences through the CUDA residual,
bitwise reproducibility, and the torch.autograd.Function."""

import numpy as np
import pytest
import torch

import oracle
import paper_1607_04245_gb300 as fem
import workloads
from gpu_util import TOL, as_input, device_arrays, rel_err, residual, to_dev
from paper_1607_04245_gb300.autograd import DeviceMesh, laplacian_residual

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def adj3d():
    return workloads.adjoint_case()  # 1,572,864 tets


def _lists_ok(conn_np, V, ptr, idx):
    ptr = ptr.cpu().numpy().astype(np.int64)
    idx = idx.cpu().numpy().astype(np.int64)
    nb, C = conn_np.shape
    deg = np.bincount(conn_np.ravel(), minlength=V)
    assert ptr[0] == 0 and np.array_equal(np.diff(ptr), deg)
    cell, a = idx // nb, idx % nb
    owner = np.repeat(np.arange(V), deg)
    assert np.array_equal(conn_np[a, cell], owner)  # every entry points back at its vertex
    assert np.all(np.diff(idx)[np.diff(owner) == 0] > 0)  # sorted within each vertex
    assert np.array_equal(np.sort(idx), np.arange(nb * C))  # each (cell, vertex) exactly once


@pytest.mark.parametrize("dim,n_cells", [(2, 8192), (3, 3071), (3, 1572864)])
def test_node2cell_lists(dim, n_cells):
    case = workloads.laplacian_square_case() if dim == 2 else workloads.laplacian_cube_case(n_cells)
    conn = to_dev(case.mesh.conn, torch.int32)
    ptr, idx = fem.fem_build_node2cell(conn, case.n_verts)
    torch.cuda.synchronize()
    _lists_ok(case.mesh.conn, case.n_verts, ptr, idx)


def _adjoint(c, d, prec, mesh=None):
    q = c.rule
    if mesh is None:
        ptr, idx = fem.fem_build_node2cell(d["conn"], c.n_verts)
    else:
        ptr, idx = mesh.node_ptr, mesh.node_idx
    return fem.fem_adjoint_laplacian(d["coords"], d["conn"], d["u"], d["K"], q.points, q.weights, d["adj"], ptr, idx,
                                     prec=prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_parity_full(adj3d, prec):
    c, d = device_arrays(adj3d, prec)
    dK, du = _adjoint(c, d, prec)
    torch.cuda.synchronize()
    rK, ru = oracle.adjoint_for(c)
    eK, eu = rel_err(dK, rK), rel_err(du, ru)
    print(f"adjoint {prec}: dK err {eK:.3e}, du err {eu:.3e}")
    assert eK <= TOL[prec] and eu <= TOL[prec]
    if prec == "mixed":
        rK64, ru64 = oracle.adjoint_for(adj3d)  # the unrounded float64 u, K and lambda
        eK64, eu64 = rel_err(dK, rK64), rel_err(du, ru64)
        print(f"adjoint mixed vs the float64 inputs: dK {eK64:.3e}, du {eu64:.3e}")
        assert eK64 <= TOL["mixed"] and eu64 <= TOL["mixed"]


@pytest.mark.parametrize("n_cells", [1, 5, 6 * 6 ** 3 - 2])
@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_adjoint_ragged(n_cells, prec):
    case = workloads.adjoint_case(n_cells)
    c, d = device_arrays(case, prec)
    dK, du = _adjoint(c, d, prec)
    torch.cuda.synchronize()
    rK, ru = oracle.adjoint_for(c)
    assert rel_err(dK, rK) <= TOL[prec] and rel_err(du, ru) <= TOL[prec]


def test_adjoint_2d():
    case = workloads.laplacian_square_case()
    case.adj = np.random.default_rng(5).uniform(-1, 1, (3, case.n_cells))
    for prec in ("fp64", "mixed"):
        c, d = device_arrays(case, prec)
        dK, du = _adjoint(c, d, prec)
        torch.cuda.synchronize()
        rK, ru = oracle.adjoint_for(c)
        assert rel_err(dK, rK) <= TOL[prec] and rel_err(du, ru) <= TOL[prec]


def test_adjoint_bitwise_reproducible(adj3d):
    c, d = device_arrays(adj3d, "mixed")
    dK1, du1 = _adjoint(c, d, "mixed")
    dK2, du2 = _adjoint(c, d, "mixed")
    torch.cuda.synchronize()
    assert torch.equal(dK1, dK2) and torch.equal(du1, du2)


def test_central_differences_64_directions(adj3d):
    """J(u, K) = sum lambda . r(u, K) through the CUDA float64 residual; h = 1e-6, seeds 1..64."""
    c, d = device_arrays(adj3d, "fp64")
    dK, du = _adjoint(c, d, "fp64")
    lam = d["adj"]

    def J(u, K):
        r = fem.fem_integrate_laplacian(d["coords"], d["conn"], u, K, c.rule.points, c.rule.weights, prec="fp64")
        return float((lam * r).sum().item())

    h = 1e-6
    worst = 0.0
    for s in range(1, 65):
        g = torch.Generator(device="cuda").manual_seed(s)
        dKd = torch.randn(d["K"].shape, generator=g, device="cuda", dtype=torch.float64)
        dud = torch.randn(d["u"].shape, generator=g, device="cuda", dtype=torch.float64)
        fd = (J(d["u"] + h * dud, d["K"] + h * dKd) - J(d["u"] - h * dud, d["K"] - h * dKd)) / (2 * h)
        an = float((dK * dKd).sum().item() + (du * dud).sum().item())
        worst = max(worst, abs(fd - an) / max(abs(an), 1e-300))
    print(f"central differences: worst relative deviation {worst:.3e}")
    assert worst <= 1e-6


def test_autograd_function_matches_oracle():
    case = workloads.adjoint_case(6 * 8 ** 3)
    c, d = device_arrays(case, "fp64")
    mesh = DeviceMesh(d["coords"], d["conn"], c.rule.points, c.rule.weights)
    u = d["u"].clone().requires_grad_(True)
    K = d["K"].clone().requires_grad_(True)
    r = laplacian_residual(u, K, mesh, "fp64")
    (r * d["adj"]).sum().backward()
    rK, ru = oracle.adjoint_for(c)
    assert rel_err(K.grad, rK) <= TOL["fp64"]
    assert rel_err(u.grad, ru) <= TOL["fp64"]
    assert rel_err(r.detach(), oracle.residual_for(c)) <= TOL["fp64"]


def test_autograd_gradcheck_small():
    case = workloads.laplacian_cube_case(6 * 2 ** 3)
    c, d = device_arrays(case, "fp64")
    mesh = DeviceMesh(d["coords"], d["conn"], c.rule.points, c.rule.weights)
    u = d["u"].clone().requires_grad_(True)
    K = d["K"].clone().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda uu, KK: laplacian_residual(uu, KK, mesh, "fp64"), (u, K),
                                    eps=1e-6, atol=1e-8, rtol=1e-6)
