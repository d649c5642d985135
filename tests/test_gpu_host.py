"""The host-buffer entry (fem_integrate_laplacian_host: chunked, overlapped copies, or with
chunks = 0 the kernel reading and writing the page-locked host arrays directly) gives the
same element vectors as the device entry, and matches the oracle."""

import numpy as np
import pytest
import torch

import oracle
import paper_1607_04245_gb300 as fem
import workloads
from gpu_util import TOL, device_arrays, rel_err
from paper_1607_04245_gb300.host import HostIntegrator

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,n_cells", [(2, 8192), (3, 6 * 24 ** 3), (3, 6 * 24 ** 3 - 2), (3, 5)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("chunks", [0, 1, 3, 8])
def test_host_path_equals_device_path(dim, n_cells, prec, chunks):
    base = workloads.laplacian_square_case() if dim == 2 else workloads.laplacian_cube_case(6 * 24 ** 3)
    mesh = workloads.first_cells(base.mesh, n_cells)
    case = workloads.Case("laplacian", mesh, base.rule, base.u[: mesh.n_verts], K=base.K[:, :n_cells].copy())
    c, d = device_arrays(case, prec)
    ref_dev = fem.fem_integrate_laplacian(d["coords"], d["conn"], d["u"], d["K"], c.rule.points, c.rule.weights,
                                          prec=prec).cpu()
    dt = fem.value_dtype(prec)
    hi = HostIntegrator("cuda")
    out = hi.laplacian(hi.pinned("coords", c.mesh.coords, torch.float64), hi.pinned("conn", c.mesh.conn, torch.int32),
                       hi.pinned("u", c.u, dt), hi.pinned("K", c.K, dt), c.rule.points, c.rule.weights, prec=prec,
                       chunks=chunks)
    hi.stream.synchronize()
    if prec == "fp64" or (n_cells % 4 == 0 and chunks > 0):
        # every chunk runs the kernel the device entry runs on the whole mesh: same bits
        assert torch.equal(out, ref_dev)
    else:
        # the ragged last chunk, or (chunks = 0) the plain-load kernel, computes one cell
        # per call of the scalar float32 routine, the device entry's pair kernel two
        assert rel_err(out, ref_dev.double().numpy()) <= 1e-6
    assert rel_err(out, oracle.residual_for(c)) <= TOL[prec]


def test_host_path_rejects_small_workspace():
    case = workloads.laplacian_square_case(8)
    dt = torch.float64
    t = lambda a, ty: torch.from_numpy(np.ascontiguousarray(a)).to(ty)
    out = torch.empty((3, case.n_cells), dtype=dt)
    with pytest.raises(fem.FemError):
        fem.fem_integrate_laplacian_host(t(case.mesh.coords, dt), t(case.mesh.conn, torch.int32), t(case.u, dt),
                                         t(case.K, dt), case.rule.points, case.rule.weights, out,
                                         torch.empty(64, dtype=torch.uint8, device="cuda"), prec="fp64")


def test_host_path_mapped_rejects_pageable_memory():
    """chunks = 0 needs page-locked host arrays; pageable ones are an argument error, not
    a kernel access."""
    case = workloads.laplacian_square_case(8)
    dt = torch.float64
    t = lambda a, ty: torch.from_numpy(np.ascontiguousarray(a)).to(ty)
    out = torch.empty((3, case.n_cells), dtype=dt)
    need = fem.fem_host_work_bytes(2, case.n_cells, case.mesh.n_verts, case.rule.n_q, "fp64", chunks=0)
    work = torch.empty(need, dtype=torch.uint8, device="cuda")
    with pytest.raises(fem.FemError):
        fem.fem_integrate_laplacian_host(t(case.mesh.coords, dt), t(case.mesh.conn, torch.int32), t(case.u, dt),
                                         t(case.K, dt), case.rule.points, case.rule.weights, out, work, chunks=0,
                                         prec="fp64")
    torch.cuda.synchronize()
