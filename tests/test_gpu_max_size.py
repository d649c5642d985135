"""The largest mesh the int32 indexing admits: (dim+1) * n_cells < 2^31, i.e. 536,870,911
tetrahedra in 3D (about 26 GB of cell data in the float32 forms, 43 GB in float64).

The connectivity and coefficient rows are the 1,572,864-tet workload repeated over the
whole range (the same vertex set), so every cell's element vector must equal the one of
its counterpart in the base workload: bit for bit on the paths that compute a cell the
same way at any position (the float32 forms' pair kernel and the float64 form's staged
kernel on a size divisible by 4, every float64 path),
within the float32 tolerance on the ragged size, and against the oracle on a sample of
cells spread over the whole range. One more cell is refused on the host.
"""

import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1607_04245_gb300 as fem
import workloads
from gpu_util import TOL, device_arrays

pytestmark = pytest.mark.gpu

C_MAX = ((1 << 31) - 1) // 4  # 536,870,911 tetrahedra


@pytest.fixture(scope="module")
def base():
    return workloads.laplacian_cube_case()


def _tile(rows: torch.Tensor, n: int) -> torch.Tensor:
    """rows [r][C0] repeated along the cell axis to [r][n]."""
    r, c0 = rows.shape
    big = torch.empty((r, n), dtype=rows.dtype, device=rows.device)
    k = n // c0
    big[:, : k * c0].view(r, k, c0).copy_(rows[:, None, :].expand(r, k, c0))
    big[:, k * c0:] = rows[:, : n - k * c0]
    return big


def _same_as_tiled(out: torch.Tensor, ref: torch.Tensor) -> bool:
    n, c0 = out.shape[1], ref.shape[1]
    k = n // c0
    ok = bool(torch.equal(out[:, : k * c0].view(out.shape[0], k, c0), ref[:, None, :].expand(-1, k, -1)))
    return ok and bool(torch.equal(out[:, k * c0:], ref[:, : n - k * c0]))


def _max_rel_dev_from_tiled(out: torch.Tensor, ref: torch.Tensor) -> float:
    n, c0 = out.shape[1], ref.shape[1]
    k = n // c0
    worst = 0.0
    for i in range(k + 1):  # one block at a time: no 2 G-element temporaries
        a, b = i * c0, min(n, (i + 1) * c0)
        if a >= b:
            break
        d = (out[:, a:b].double() - ref[:, : b - a].double()).abs().max().item()
        worst = max(worst, d)
    return worst / ref.double().abs().max().item()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_max_size_equals_tiled_base(base, prec):
    c, d = device_arrays(base, prec)
    q = c.rule
    ref = fem.fem_integrate_laplacian(d["coords"], d["conn"], d["u"], d["K"], q.points, q.weights, prec=prec)
    ref_ora = oracle.residual_for(c)
    c0 = c.n_cells
    scale = np.abs(ref_ora).max()
    rng = np.random.default_rng(0)
    for n in (C_MAX - C_MAX % 4, C_MAX):
        # n divisible by 4: the pair kernel (float32 forms) or the staged kernel (float64);
        # n = C_MAX (ragged): the
        # scalar-load kernel, whose float32 cells go one per call instead of in pairs, so
        # only its float64 form is bitwise the tiled base
        conn, K = _tile(d["conn"], n), _tile(d["K"], n)
        out = fem.fem_integrate_laplacian(d["coords"], conn, d["u"], K, q.points, q.weights, prec=prec)
        torch.cuda.synchronize()
        del conn, K
        if n % 4 == 0 or prec == "fp64":
            assert _same_as_tiled(out, ref)
        else:
            assert _max_rel_dev_from_tiled(out, ref) <= 1e-6
        # a sample of cells over the whole range, and both ends, against the oracle
        cells = np.concatenate([rng.integers(0, n, 4096), [0, n - 1]])
        got = out[:, torch.from_numpy(cells).to(out.device)].double().cpu().numpy()
        assert np.abs(got - ref_ora[:, cells % c0]).max() / scale <= TOL[prec]
        assert fem.fem_device_error() == 0
        del out
        torch.cuda.empty_cache()


def test_one_cell_more_is_refused(base):
    """(dim+1) * n_cells = 2^31: FEM_ERR_SHAPE from the host-side check, before any launch
    (the arrays passed are the small base ones; the library does not touch them)."""
    c, d = device_arrays(base, "fp64")
    q = c.rule
    out = torch.empty((4, 8), dtype=torch.float64, device="cuda")
    qp = np.ascontiguousarray(q.points, dtype=np.float64)
    qw = np.ascontiguousarray(q.weights, dtype=np.float64)
    P = ctypes.c_void_p
    L = fem.binding.lib()
    st = L.fem_integrate_laplacian(3, C_MAX + 1, c.mesh.n_verts, P(d["coords"].data_ptr()),
                                   P(d["conn"].data_ptr()), P(d["u"].data_ptr()), P(d["K"].data_ptr()), q.n_q,
                                   qp.ctypes.data_as(P), qw.ctypes.data_as(P), P(out.data_ptr()),
                                   fem.binding.precision("fp64"), None)
    assert st == -2  # FEM_ERR_SHAPE
    assert b"int32" in L.fem_last_error()


def test_elasticity_max_size_mixed():
    """3D elasticity at the largest cell count the int32 indexing admits (12 output rows of
    536,870,908 cells, 51 GB in all): the 2^21-tet workload's rows repeated, every element
    vector bitwise its base counterpart, a sample against the oracle."""
    base = workloads.elasticity_case(3)
    c, d = device_arrays(base, "mixed")
    q = c.rule
    ref = fem.fem_integrate_elasticity(d["coords"], d["conn"], d["u"], d["lam"], d["mu"], q.points, q.weights,
                                       prec="mixed")
    ref_ora = oracle.residual_for(c)
    n = C_MAX - C_MAX % 4
    conn, lam, mu = _tile(d["conn"], n), _tile(d["lam"], n), _tile(d["mu"], n)
    out = fem.fem_integrate_elasticity(d["coords"], conn, d["u"], lam, mu, q.points, q.weights, prec="mixed")
    torch.cuda.synchronize()
    del conn, lam, mu
    try:
        assert _same_as_tiled(out, ref)
        rng = np.random.default_rng(1)
        cells = np.concatenate([rng.integers(0, n, 4096), [0, n - 1]])
        got = out[:, torch.from_numpy(cells).to(out.device)].double().cpu().numpy()
        assert np.abs(got - ref_ora[:, cells % c.n_cells]).max() / np.abs(ref_ora).max() <= TOL["mixed"]
        assert fem.fem_device_error() == 0
    finally:
        del out
        torch.cuda.empty_cache()
