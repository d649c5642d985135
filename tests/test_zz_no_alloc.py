"""fem_adjoint_laplacian_noalloc: the adjoint for callers that cannot allocate device
memory (a plugin or callback handed only input and output pointers, or a loop that
must avoid cudaMalloc's device-wide synchronisation). Its workspace is a fixed array
inside the library, so it takes no scratch argument.

Called here through the C ABI (ctypes, raw device pointers) and compared with
fem_adjoint_laplacian, which takes a caller-owned workspace, on two calls in a row with
different adjoint weights: the second call reuses the array the first one wrote. Both
entry points run the same kernels, so the results must be bitwise equal; a stale entry
left in the array by an earlier, larger call would show up as a difference. One call is
also checked against the CPU oracle. This file is named to be collected last; it also
passes on its own in a fresh process.
"""

import oracle

import ctypes

import numpy as np
import pytest
import torch

import paper_1607_04245_gb300 as fem
import workloads
from gpu_util import TOL, device_arrays, rel_err
from paper_1607_04245_gb300 import binding

pytestmark = pytest.mark.gpu


def _noalloc(c, d, lam, ptr, idx, prec):
    L = binding.lib()
    f = L.fem_adjoint_laplacian_noalloc
    P, i64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    f.argtypes = [ci, i64, i64, P, P, P, P, ci, P, P, P, P, P, P, P, ci, P]
    f.restype = ci
    dt = fem.value_dtype(prec)
    dK = torch.full((c.rule.n_q, c.n_cells), float("nan"), dtype=dt, device="cuda")
    du = torch.full((c.n_verts,), float("nan"), dtype=dt, device="cuda")
    qp = np.ascontiguousarray(c.rule.points)
    qw = np.ascontiguousarray(c.rule.weights)
    st = f(c.dim, c.n_cells, c.n_verts, d["coords"].data_ptr(), d["conn"].data_ptr(), d["u"].data_ptr(),
           d["K"].data_ptr(), c.rule.n_q, qp.ctypes.data, qw.ctypes.data, lam.data_ptr(), dK.data_ptr(),
           du.data_ptr(), ptr.data_ptr(), idx.data_ptr(), binding.precision(prec),
           torch.cuda.current_stream().cuda_stream)
    assert st == 0, L.fem_last_error().decode()
    return dK, du


@pytest.mark.parametrize("dim,prec", [(3, "fp64"), (3, "mixed"), (2, "mixed")])
def test_noalloc_matches_workspace_entry_point_twice(dim, prec):
    case = workloads.adjoint_case(6 * 40 ** 3) if dim == 3 else workloads.laplacian_square_case(256)
    c, d = device_arrays(case, prec)
    ptr, idx = fem.fem_build_node2cell(d["conn"], c.n_verts)
    dt = fem.value_dtype(prec)
    rng = np.random.default_rng(42)
    for call in range(2):
        lam = torch.from_numpy(rng.uniform(-1, 1, (dim + 1, c.n_cells))).to("cuda", dt)
        dK, du = _noalloc(c, d, lam, ptr, idx, prec)
        rK, ru = fem.fem_adjoint_laplacian(d["coords"], d["conn"], d["u"], d["K"], c.rule.points, c.rule.weights,
                                           lam, ptr, idx, prec=prec)
        torch.cuda.synchronize()
        assert fem.fem_device_error() == 0
        assert torch.equal(dK, rK), (call, "dK")
        assert torch.equal(du, ru), (call, "du")
        if call == 1:
            oK, ou = oracle.adjoint_for(c, lam.double().cpu().numpy())
            assert rel_err(dK, oK) <= TOL[prec] and rel_err(du, ou) <= TOL[prec]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_noalloc_large_call_then_small_call(prec):
    """A call that fills most of the array, then a smaller one on another mesh: the
    smaller call must not read anything the larger one left behind."""
    dt = fem.value_dtype(prec)
    rng = np.random.default_rng(3)
    for n in (6 * 40 ** 3, 6 * 9 ** 3 + 6):
        case = workloads.adjoint_case(n)
        c, d = device_arrays(case, prec)
        ptr, idx = fem.fem_build_node2cell(d["conn"], c.n_verts)
        lam = torch.from_numpy(rng.uniform(-1, 1, (4, c.n_cells))).to("cuda", dt)
        dK, du = _noalloc(c, d, lam, ptr, idx, prec)
        rK, ru = fem.fem_adjoint_laplacian(d["coords"], d["conn"], d["u"], d["K"], c.rule.points, c.rule.weights,
                                           lam, ptr, idx, prec=prec)
        torch.cuda.synchronize()
        assert torch.equal(dK, rK) and torch.equal(du, ru), n


def test_noalloc_double_float_form():
    """FEM_FP64_DF through the fixed array: float64 values, 8 bytes per workspace entry."""
    case = workloads.adjoint_case(6 * 24 ** 3)
    c, d = device_arrays(case, "fp64")
    ptr, idx = fem.fem_build_node2cell(d["conn"], c.n_verts)
    lam = torch.from_numpy(np.random.default_rng(7).uniform(-1, 1, (4, c.n_cells))).to("cuda", torch.float64)
    dK, du = _noalloc(c, d, lam, ptr, idx, "fp64_df")
    rK, ru = fem.fem_adjoint_laplacian(d["coords"], d["conn"], d["u"], d["K"], c.rule.points, c.rule.weights, lam,
                                       ptr, idx, prec="fp64_df")
    assert torch.equal(dK, rK) and torch.equal(du, ru)


def test_noalloc_rejects_sizes_beyond_its_array():
    L = binding.lib()
    f = L.fem_adjoint_laplacian_noalloc
    P, i64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    f.argtypes = [ci, i64, i64, P, P, P, P, ci, P, P, P, P, P, P, P, ci, P]
    f.restype = ci
    limit = 16 << 20
    too_many = limit // (4 * 8) + 1  # 3D float64: 4 values of 8 bytes per cell
    qw = np.full(4, 1 / 24)
    st = f(3, too_many, 10, None, None, None, None, 4, None, qw.ctypes.data, None, None, None, None, None, 0, None)
    assert st == -2
    assert b"fixed" in L.fem_last_error()
