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


def test_prepare_option_launches_the_plain_call():
    """prepare=True returns the call as a PreparedCall; running it gives bitwise what the
    plain call gives (adjoint, reaction-diffusion, precomputed geometry, prepared records,
    several fields, run-time compiled physics)."""
    case = workloads.adjoint_case(24576).rounded_to_f32()
    f32 = torch.float32
    coords, conn = to_dev(case.mesh.coords, torch.float64), to_dev(case.mesh.conn, torch.int32)
    u, K, q, V, C = to_dev(case.u, f32), to_dev(case.K, f32), case.rule, case.n_verts, case.n_cells
    lam = to_dev(case.adj, f32)
    ptr, idx = fem.fem_build_node2cell(conn, V)
    a = torch.linspace(0.5, 2.0, V, device="cuda", dtype=f32)
    cr = torch.linspace(0.25, 1.0, q.n_q * C, device="cuda", dtype=f32).reshape(q.n_q, C)
    geom = fem.fem_precompute_geometry(coords, conn)
    rec = fem.fem_prepare_vertices(coords)
    U = torch.stack([u, -u, 2 * u])
    calls = {
        "adjoint": (lambda **k: fem.fem_adjoint_laplacian(coords, conn, u, K, q.points, q.weights, lam, ptr, idx, **k),
                    lambda: dict(dK=torch.empty((q.n_q, C), dtype=f32, device="cuda"),
                                 du=torch.empty(V, dtype=f32, device="cuda"))),
        "reaction": (lambda **k: fem.fem_integrate_reaction_diffusion(coords, conn, u, a, q.points, q.weights, c=cr,
                                                                      a_space=1, drift=1.0, **k),
                     lambda: dict(out=torch.empty((4, C), dtype=f32, device="cuda"))),
        "geom": (lambda **k: fem.fem_integrate_laplacian_geom(conn, V, u, K, q.points, q.weights, geom, **k),
                 lambda: dict(out=torch.empty((4, C), dtype=f32, device="cuda"))),
        "prepared": (lambda **k: fem.fem_integrate_laplacian_prepared(coords, rec, conn, u, K, q.points, q.weights,
                                                                      **k),
                     lambda: dict(out=torch.empty((4, C), dtype=f32, device="cuda"))),
        "fields": (lambda **k: fem.fem_integrate_laplacian_fields(coords, conn, U, K, q.points, q.weights, **k),
                   lambda: dict(out=torch.empty((3, 4, C), dtype=f32, device="cuda"))),
        "pointwise": (lambda **k: fem.fem_integrate_pointwise(coords, conn, u, K[None].contiguous(), q.points,
                                                              q.weights, f1="for (int i = 0; i < DIM; ++i) "
                                                              "f1[i] = a[0] * grad_u[i];", **k),
                      lambda: dict(out=torch.empty((4, C), dtype=f32, device="cuda"))),
    }
    for name, (call, outs) in calls.items():
        o1, o2 = outs(), outs()
        call(**o1)
        pc = call(prepare=True, **o2)
        assert isinstance(pc, fem.PreparedCall), name
        torch.cuda.synchronize()
        pc()
        pc()
        torch.cuda.synchronize()
        for k in o1:
            assert torch.equal(o1[k], o2[k]), (name, k)


def test_run_time_compiled_kernel_in_an_unsynchronised_chain():
    """The kernel fem_integrate_pointwise generates also waits for the kernel before it: a
    chain of its residuals and assemblies with no synchronisation equals the synchronised
    chain bitwise."""
    case = workloads.laplacian_cube_case(196608).rounded_to_f32()
    f32 = torch.float32
    coords, conn = to_dev(case.mesh.coords, torch.float64), to_dev(case.mesh.conn, torch.int32)
    V, q = case.n_verts, case.rule
    K = to_dev(case.K, f32)[None].contiguous()
    ptr, idx = fem.fem_build_node2cell(conn, V)
    f1 = "for (int i = 0; i < DIM; ++i) f1[i] = a[0] * grad_u[i];"

    def chain(sync):
        u = to_dev(case.u, f32).reshape(1, V)
        fields = [u]
        elem = torch.empty((4, case.n_cells), dtype=f32, device="cuda")
        torch.cuda.synchronize()
        for _ in range(STEPS):
            fem.fem_integrate_pointwise(coords, conn, fields[-1][0], K, q.points, q.weights, f1=f1, out=elem,
                                        prec="mixed")
            if sync:
                torch.cuda.synchronize()
            nxt = torch.empty((1, V), dtype=f32, device="cuda")
            fem.fem_gather_nodes(elem, ptr, idx, V, 3, out=nxt, prec="mixed")
            if sync:
                torch.cuda.synchronize()
            fields.append(nxt)
        torch.cuda.synchronize()
        return fields

    a, b = chain(False), chain(True)
    assert fem.fem_device_error() == 0
    for i, (x, y) in enumerate(zip(a, b)):
        assert torch.equal(x, y), i
    assert not torch.equal(a[-1], a[-2])


@pytest.mark.parametrize("kind", ("geom", "reaction", "prepared"))
def test_other_overlapped_kernels_in_an_unsynchronised_chain(kind):
    """The precomputed-geometry, reaction-diffusion and prepared-record kernels in a
    dependent chain with the gather kernel, unsynchronised against synchronised."""
    case = workloads.laplacian_cube_case(196608).rounded_to_f32()
    f32 = torch.float32
    coords, conn = to_dev(case.mesh.coords, torch.float64), to_dev(case.mesh.conn, torch.int32)
    V, C, q = case.n_verts, case.n_cells, case.rule
    K = to_dev(case.K, f32)
    ptr, idx = fem.fem_build_node2cell(conn, V)
    geom = fem.fem_precompute_geometry(coords, conn)
    rec = fem.fem_prepare_vertices(coords)
    a = torch.linspace(0.5, 2.0, V, device="cuda", dtype=f32)
    cr = torch.linspace(0.25, 1.0, q.n_q * C, device="cuda", dtype=f32).reshape(q.n_q, C)

    def step(v, out):
        if kind == "geom":
            fem.fem_integrate_laplacian_geom(conn, V, v, K, q.points, q.weights, geom, out=out)
        elif kind == "reaction":
            fem.fem_integrate_reaction_diffusion(coords, conn, v, a, q.points, q.weights, c=cr, a_space=1,
                                                 drift=1.0, out=out)
        else:
            fem.fem_integrate_laplacian_prepared(coords, rec, conn, v, K, q.points, q.weights, out=out)

    def chain(sync):
        fields = [to_dev(case.u, f32).reshape(1, V)]
        elem = torch.empty((4, C), dtype=f32, device="cuda")
        torch.cuda.synchronize()
        for _ in range(STEPS):
            step(fields[-1][0], elem)
            if sync:
                torch.cuda.synchronize()
            nxt = torch.empty((1, V), dtype=f32, device="cuda")
            fem.fem_gather_nodes(elem, ptr, idx, V, 3, out=nxt, prec="mixed")
            if sync:
                torch.cuda.synchronize()
            fields.append(nxt)
        torch.cuda.synchronize()
        return fields

    x, y = chain(False), chain(True)
    assert fem.fem_device_error() == 0
    for i, (p, r) in enumerate(zip(x, y)):
        assert torch.equal(p, r), (kind, i)
    assert not torch.equal(x[-1], x[-2])
