"""Launches that overlap the tail of the kernel before them (programmatic dependent launch).

Each library kernel launched that way waits, before its first global memory access, until
the kernel before it on the stream has completed and its writes are visible. A chain of
dependent calls -- a residual, the assembly E^T of its element vectors into the next
nodal field, the residual of that field, ... -- enqueued with no synchronisation between
the calls must therefore give bitwise the fields of the same chain synchronised after
every call. The chain runs the float32 pair kernel, the float64 staged kernel, the
double-float kernels, the elasticity kernels and the gather kernel back to back.

Also: a PreparedCall (arguments marshalled once) launches exactly what the plain call
launches."""

import pytest
import torch

import paper_1607_04245_gb300 as fem
import workloads
from gpu_util import to_dev

pytestmark = pytest.mark.gpu

STEPS = 8


def _chain(case, prec, sync):
    c = case if prec in ("fp64", "fp64_df") else case.rounded_to_f32()
    dt = fem.value_dtype(prec)
    coords, conn = to_dev(c.mesh.coords, torch.float64), to_dev(c.mesh.conn, torch.int32)
    V, dim, q = c.n_verts, c.dim, c.rule
    ptr, idx = fem.fem_build_node2cell(conn, V)
    if c.physics == "laplacian":
        u, K = to_dev(c.u, dt).reshape(1, V), to_dev(c.K, dt)
        step = lambda v, out: fem.fem_integrate_laplacian(coords, conn, v[0], K, q.points, q.weights, out=out,
                                                          prec=prec)
    else:
        u, lam, mu = to_dev(c.u, dt), to_dev(c.lam, dt), to_dev(c.mu, dt)
        step = lambda v, out: fem.fem_integrate_elasticity(coords, conn, v, lam, mu, q.points, q.weights, out=out,
                                                           prec=prec)
    torch.cuda.synchronize()
    fields = [u]
    elem = torch.empty(((dim + 1) * c.n_comp, c.n_cells), dtype=dt, device="cuda")
    for _ in range(STEPS):
        step(fields[-1], elem)
        if sync:
            torch.cuda.synchronize()
        nxt = torch.empty((c.n_comp, V), dtype=dt, device="cuda")
        fem.fem_gather_nodes(elem, ptr, idx, V, dim, out=nxt, prec=prec)
        if sync:
            torch.cuda.synchronize()
        fields.append(nxt)
    torch.cuda.synchronize()
    return fields


CASES = [("laplacian", "fp64"), ("laplacian", "mixed"), ("laplacian", "fp32"), ("laplacian", "fp64_df"),
         ("elasticity", "mixed"), ("elasticity", "fp64"), ("elasticity", "fp64_df")]


@pytest.mark.parametrize("physics,prec", CASES)
def test_unsynchronised_dependent_chain_equals_synchronised(physics, prec):
    case = (workloads.laplacian_cube_case(196608) if physics == "laplacian"
            else workloads.elasticity_case(3, 196608))
    a = _chain(case, prec, sync=False)
    b = _chain(case, prec, sync=True)
    assert fem.fem_device_error() == 0
    for i, (x, y) in enumerate(zip(a, b)):
        assert torch.equal(x, y), (physics, prec, i)
    # the chain does change the field at every step (each step reads the previous one)
    assert not torch.equal(a[-1], a[-2])


@pytest.mark.parametrize("prec", ("mixed", "fp64", "fp64_df"))
def test_prepared_call_launches_the_plain_call(prec):
    case = workloads.laplacian_cube_case(24576)
    c = case if prec in ("fp64", "fp64_df") else case.rounded_to_f32()
    dt = fem.value_dtype(prec)
    coords, conn = to_dev(c.mesh.coords, torch.float64), to_dev(c.mesh.conn, torch.int32)
    u, K, q = to_dev(c.u, dt), to_dev(c.K, dt), c.rule
    ref = fem.fem_integrate_laplacian(coords, conn, u, K, q.points, q.weights, prec=prec)
    out = torch.full_like(ref, float("nan"))
    call = fem.prepared_integrate_laplacian(coords, conn, u, K, q.points, q.weights, out, prec=prec)
    call()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    out.fill_(float("nan"))
    call()
    call()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    el = workloads.elasticity_case(3, 24576)
    e = el if prec in ("fp64", "fp64_df") else el.rounded_to_f32()
    args = (coords, conn) if e.n_verts == c.n_verts else (to_dev(e.mesh.coords, torch.float64),
                                                          to_dev(e.mesh.conn, torch.int32))
    ue, lam, mu = to_dev(e.u, dt), to_dev(e.lam, dt), to_dev(e.mu, dt)
    ref = fem.fem_integrate_elasticity(*args, ue, lam, mu, e.rule.points, e.rule.weights, prec=prec)
    out = torch.full_like(ref, float("nan"))
    fem.prepared_integrate_elasticity(*args, ue, lam, mu, e.rule.points, e.rule.weights, out, prec=prec)()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


def test_prepared_call_validates_once_at_preparation():
    case = workloads.laplacian_cube_case(6000).rounded_to_f32()
    coords, conn = to_dev(case.mesh.coords, torch.float64), to_dev(case.mesh.conn, torch.int32)
    u, K, q = to_dev(case.u, torch.float32), to_dev(case.K, torch.float32), case.rule
    bad_out = torch.empty((3, case.n_cells), dtype=torch.float32, device="cuda")  # dim+1 = 4 rows needed
    with pytest.raises(ValueError):
        fem.prepared_integrate_laplacian(coords, conn, u, K, q.points, q.weights, bad_out)
