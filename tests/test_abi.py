"""The C-ABI library loads, exports every function include/fem.h declares, and its
host-side argument checks return the documented statuses. No kernel is launched:
every call here fails validation (or is a no-op) before touching a GPU."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_1607_04245_gb300 import build as fem_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    fem_build.build()
    from paper_1607_04245_gb300 import binding

    return binding.lib()


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(fem_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fem_integrate_laplacian", "fem_integrate_elasticity", "fem_adjoint_laplacian",
                     "fem_build_node2cell", "fem_status_string", "fem_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    for st in (0, -1, -2, -3, -4, -5, -6, -7):
        assert lib.fem_status_string(st)
    assert b"sm_103a" in lib.fem_version()


def _qw(n):
    return np.full(n, 1.0 / (2 * n))


def test_host_validation(lib):
    P = ctypes.c_void_p
    qw = _qw(3)
    qwp = qw.ctypes.data_as(P)
    fake = P(0x1000)  # never dereferenced: validation fails or the call is a no-op first
    # dim outside {2, 3}
    assert lib.fem_integrate_laplacian(4, 10, 10, fake, fake, fake, fake, 3, None, qwp, fake, 0, None) == -1
    # negative size
    assert lib.fem_integrate_laplacian(2, -1, 10, fake, fake, fake, fake, 3, None, qwp, fake, 0, None) == -1
    # n_q out of range
    assert lib.fem_integrate_laplacian(2, 10, 10, fake, fake, fake, fake, 0, None, qwp, fake, 0, None) == -2
    assert lib.fem_integrate_laplacian(2, 10, 10, fake, fake, fake, fake, 33, None, qwp, fake, 0, None) == -2
    # NULL weights
    assert lib.fem_integrate_laplacian(2, 10, 10, fake, fake, fake, fake, 3, None, None, fake, 0, None) == -1
    # quadrature point outside the reference triangle
    bad = np.array([[0.5, 0.6], [0.1, 0.1], [0.2, 0.2]])
    assert lib.fem_integrate_laplacian(2, 10, 10, fake, fake, fake, fake, 3, bad.ctypes.data_as(P), qwp, fake, 0,
                                       None) == -1
    # unknown precision
    assert lib.fem_integrate_laplacian(2, 10, 10, fake, fake, fake, fake, 3, None, qwp, fake, 7, None) == -1
    # too large for int32 indexing
    assert lib.fem_integrate_laplacian(3, 1 << 30, 10, fake, fake, fake, fake, 3, None, qwp, fake, 0, None) == -2
    assert b"int32" in lib.fem_last_error()
    # NULL output
    assert lib.fem_integrate_elasticity(2, 10, 10, fake, fake, fake, fake, fake, 3, None, qwp, None, 0, None) == -1
    # n_cells = 0 is a valid no-op (no launch)
    assert lib.fem_integrate_laplacian(2, 0, 0, None, None, None, None, 3, None, qwp, None, 1, None) == 0
    assert lib.fem_integrate_elasticity(3, 0, 0, None, None, None, None, None, 3, None, qwp, None, 1, None) == 0


def test_mixed_threshold(lib):
    old = lib.fem_get_mixed_threshold()
    assert old == pytest.approx(0.05)
    assert lib.fem_set_mixed_threshold(ctypes.c_double(-1.0)) == -1
    assert lib.fem_set_mixed_threshold(ctypes.c_double(0.2)) == 0
    assert lib.fem_get_mixed_threshold() == pytest.approx(0.2)
    assert lib.fem_set_mixed_threshold(ctypes.c_double(old)) == 0


def test_node2cell_work_size(lib):
    assert lib.fem_node2cell_work_size(0) == 1
    assert lib.fem_node2cell_work_size(4096) == 4096 + 1 + 1
    assert lib.fem_node2cell_work_size(4097) == 4097 + 2 + 1


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1607_04245_gb300 import binding

    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="libfem.so not found"):
        binding.lib()


def test_host_work_bytes(lib):
    """Workspace sizes of the host-buffer entry (pure host arithmetic)."""
    a256 = lambda n: (n + 255) // 256 * 256
    dim, C, V, nq = 3, 1000, 300, 4
    # chunks = 0: the device copies of the vertex arrays only
    assert lib.fem_host_work_bytes(dim, C, V, nq, 1, 0) == a256(dim * V * 8) + a256(V * 4)
    assert lib.fem_host_work_bytes(dim, C, V, nq, 0, 0) == a256(dim * V * 8) + a256(V * 8)
    # chunks >= 1: plus two buffers of conn, K and out rows for one chunk (a multiple of 4 cells)
    per = (C + 3 - 1) // 3
    per = (per + 3) // 4 * 4
    want = a256(dim * V * 8) + a256(V * 4) + 2 * (a256(4 * per * 4) + a256(nq * per * 4) + a256(4 * per * 4))
    assert lib.fem_host_work_bytes(dim, C, V, nq, 1, 3) == want
    # invalid arguments
    assert lib.fem_host_work_bytes(dim, C, V, nq, 1, -1) == -1
    assert lib.fem_host_work_bytes(4, C, V, nq, 1, 1) == -1
    assert lib.fem_host_work_bytes(dim, C, V, 0, 1, 1) == -1


def test_serve_launch_validation(lib):
    """Host-side checks of the serving launcher (no CUDA call is reached)."""
    from paper_1607_04245_gb300.serving import ServeRequestDesc

    P = ctypes.c_void_p
    lib.fem_serve_launch.argtypes = [ctypes.POINTER(ServeRequestDesc), P, P, P]
    lib.fem_serve_launch.restype = ctypes.c_int
    lib.fem_serve_events_query.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.fem_serve_events_query.restype = ctypes.c_int
    fake = P(0x1000)  # never dereferenced
    assert lib.fem_serve_launch(None, fake, fake, None) == -1
    d = ServeRequestDesc()
    d.kind = 3  # no such kind
    assert lib.fem_serve_launch(ctypes.byref(d), fake, fake, None) == -1
    d.kind = 2  # the self-test: still needs a block
    assert lib.fem_serve_launch(ctypes.byref(d), fake, fake, None) == -1
    d.kind, d.physics = 1, 1  # adjoint of elasticity
    assert lib.fem_serve_launch(ctypes.byref(d), fake, fake, None) == -7
    assert lib.fem_serve_events_query(None, 0, None) == 0
    assert lib.fem_serve_events_query(None, 1, None) == -1
    lib.fem_serve_request_bytes.restype = ctypes.c_int64
    assert lib.fem_serve_request_bytes() == ctypes.sizeof(ServeRequestDesc) == 216


def test_serve_launch_checks_the_descriptor_against_its_block(lib):
    """Arrays outside the block, oversized uploads or downloads are argument errors,
    found before any copy or launch (the block pointer is never dereferenced)."""
    from paper_1607_04245_gb300.serving import SERVE_SLOTS, ServeRequestDesc

    P = ctypes.c_void_p
    lib.fem_serve_launch.argtypes = [ctypes.POINTER(ServeRequestDesc), P, P, P]
    lib.fem_serve_launch.restype = ctypes.c_int
    lib.fem_last_error.restype = ctypes.c_char_p
    fake = P(0x1000)

    def desc(C=8, V=9):
        d = ServeRequestDesc()
        d.kind, d.physics, d.dim, d.n_q, d.prec = 0, 0, 2, 3, 1
        d.n_cells, d.n_verts = C, V
        sizes = {"coords": 2 * V * 8, "conn": 3 * C * 4, "u": V * 4, "K": 3 * C * 4, "out": 3 * C * 4}
        off = 0
        for name, n in sizes.items():
            d.offset[SERVE_SLOTS[name]] = off
            off += n
        d.in_bytes = off - sizes["out"]
        d.out_bytes[0] = sizes["out"]
        d.block_bytes = off
        return d

    d = desc()
    d.block_bytes -= 1  # the element vectors end one byte past the block
    assert lib.fem_serve_launch(ctypes.byref(d), fake, fake, None) == -1
    assert b"outside" in lib.fem_last_error()
    d = desc()
    d.offset[SERVE_SLOTS["conn"]] = -16
    assert lib.fem_serve_launch(ctypes.byref(d), fake, fake, None) == -1
    d = desc()
    d.in_bytes = d.block_bytes + 1
    assert lib.fem_serve_launch(ctypes.byref(d), fake, fake, None) == -1
    d = desc()
    d.out_bytes[0] += 4
    assert lib.fem_serve_launch(ctypes.byref(d), fake, fake, None) == -1
    d = desc()
    d.out_bytes[1] = 4  # a residual request has no second result
    assert lib.fem_serve_launch(ctypes.byref(d), fake, fake, None) == -1
    d = desc()
    d.n_q = 0
    assert lib.fem_serve_launch(ctypes.byref(d), fake, fake, None) == -1

    # an adjoint request (kind 1): twelve arrays, the vertex lists' workspace last
    lib.fem_node2cell_work_size.restype = ctypes.c_int64
    lib.fem_node2cell_work_size.argtypes = [ctypes.c_int64]
    C, V = 6, 7
    sizes = {"coords": 3 * V * 8, "conn": 4 * C * 4, "u": V * 8, "K": 4 * C * 8, "adj": 4 * C * 8,
             "dK": 4 * C * 8, "du": V * 8, "scratch": 4 * C * 8, "node_ptr": (V + 1) * 4, "node_idx": 4 * C * 4,
             "work": lib.fem_node2cell_work_size(V) * 4}
    a = ServeRequestDesc()
    a.kind, a.physics, a.dim, a.n_q, a.prec = 1, 0, 3, 4, 0
    a.n_cells, a.n_verts = C, V
    off = 0
    for name, n in sizes.items():
        a.offset[SERVE_SLOTS[name]] = off
        off += n
    a.block_bytes = off - 4  # the workspace ends 4 bytes past the block
    a.out_bytes[0], a.out_bytes[1] = sizes["dK"], sizes["du"]
    assert lib.fem_serve_launch(ctypes.byref(a), fake, fake, None) == -1
    assert b"outside" in lib.fem_last_error()


def test_pointwise_validation(lib):
    """Argument checks of the run-time compiled entry point, all before any compilation."""
    P = ctypes.c_void_p
    qw = _qw(4)
    qwp = qw.ctypes.data_as(P)
    qp = np.full((4, 3), 0.25)
    qpp = qp.ctypes.data_as(P)
    fake = P(0x1000)
    f1 = b"f1[0] = grad_u[0];"
    call = lambda f0, f1, dim=3, nc=1, nk=1, nq=4, q=qpp, prec=0: lib.fem_integrate_pointwise(
        f0, f1, dim, nc, nk, 10, 10, fake, fake, fake, fake, nq, q, qwp, fake, prec, None)
    assert call(None, None) == -1  # neither f0 nor f1
    assert call(None, f1, prec=2) == -1  # FEM_FP32 ablation: not offered here
    assert call(None, f1, prec=3) == -1  # FEM_FP64_DF: not offered here
    assert call(None, f1, nc=0) == -1 and call(None, f1, nc=4) == -1
    assert call(None, f1, nk=-1) == -1 and call(None, f1, nk=9) == -1
    assert call(None, f1, dim=4) == -1
    assert call(None, f1, nq=0) == -2
    assert call(None, f1, q=None) == -1  # the quadrature points are required
    assert b"qpts" in lib.fem_last_error()


def test_serve_launch_rejects_a_status_word_the_device_cannot_reach(lib):
    """host_status must be page-locked, device-mapped host memory: plain host memory is an
    argument error found before anything is enqueued."""
    from paper_1607_04245_gb300.serving import SERVE_SLOTS, ServeRequestDesc

    P = ctypes.c_void_p
    lib.fem_serve_launch.argtypes = [ctypes.POINTER(ServeRequestDesc), P, P, P]
    lib.fem_serve_launch.restype = ctypes.c_int
    d = ServeRequestDesc()
    d.kind, d.physics, d.dim, d.n_q, d.prec, d.n_cells, d.n_verts = 2, 0, 3, 4, 1, 0, 0
    d.block_bytes = 256
    word = np.zeros(1, dtype=np.uint32)  # pageable host memory
    d.host_status = word.ctypes.data
    st = lib.fem_serve_launch(ctypes.byref(d), P(0x1000), P(0x1000), None)
    assert st in (-1, -3)  # FEM_ERR_ARG (or FEM_ERR_CUDA where no CUDA driver answers the query)


def test_serve_run_validation(lib):
    """Argument checks of the native serving loop, all made before any CUDA call."""
    from paper_1607_04245_gb300.serving import ServeRequestDesc, ServeResult

    P, i64, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    lib.fem_serve_run.argtypes = [ctypes.POINTER(ServeRequestDesc), ctypes.POINTER(i64), ctypes.POINTER(f64),
                                  ctypes.c_int, P, i64, i64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ServeResult)]
    lib.fem_serve_run.restype = ctypes.c_int
    d = (ServeRequestDesc * 2)()
    foot = (i64 * 2)(4096, 8192)
    arr = (f64 * 2)(0.0, 0.001)
    res = (ServeResult * 2)()
    pool = P(1 << 20)  # never dereferenced on the host
    run = lambda n=2, pool=pool, nbytes=1 << 20, align=256, slots=4, foot=foot, arr=arr, res=res: lib.fem_serve_run(
        d, foot, arr, n, pool, nbytes, align, slots, 1, res)
    assert run(n=0) == 0  # nothing to serve: returns at once
    assert run(slots=0) == -1 and run(slots=65) == -1
    assert run(n=-1) == -1
    assert run(pool=None) == -1 and run(res=None) == -1
    assert run(nbytes=0) == -1
    assert run(align=100) == -1 and run(align=128) == -1
    assert run(pool=P((1 << 20) + 16)) == -1  # not aligned to the arena's alignment
    assert b"aligned" in lib.fem_last_error()
    assert run(arr=(f64 * 2)(0.0, -1.0)) == -1
    assert run(arr=(f64 * 2)(0.0, float("nan"))) == -1
    assert run(foot=(i64 * 2)(4096, -1)) == -1
    assert ctypes.sizeof(ServeResult) == 32


def test_pcg_refined_validation(lib):
    """Argument checks of the refined solve, made before any CUDA call."""
    P, i64, cd, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    f = lib.fem_pcg_laplacian_refined
    f.argtypes = [ci, i64, i64, P, P, P, ci, P, P, P, P, P, P, P, ci, ci, cd, cd, P, i64, P, P, P, ci, P]
    f.restype = ci
    lib.fem_pcg_refined_work_bytes.argtypes = [ci, i64, i64, ci]
    lib.fem_pcg_refined_work_bytes.restype = i64
    fake = P(1 << 20)
    outer, inner, resid = ctypes.c_int(-1), ctypes.c_int(-1), ctypes.c_double(-1.0)
    call = lambda V=0, prec=0, rtol=1e-8, inner_rtol=1e-3, mo=5, mi=100, nq=4: f(
        3, 0, V, fake, fake, fake, nq, fake, fake, fake, fake, fake, None, fake, mo, mi, inner_rtol, rtol, fake,
        1 << 30, ctypes.byref(outer), ctypes.byref(inner), ctypes.byref(resid), prec, None)
    assert call(prec=1) == -1 and call(prec=2) == -1  # the residual runs in float64 or double-float
    assert call(inner_rtol=0.0) == -1 and call(inner_rtol=1.0) == -1
    assert call(rtol=-1.0) == -1 and call(mo=-1) == -1 and call(mi=-1) == -1
    assert call(nq=0) == -2
    assert call(V=0) == 0 and outer.value == 0 and inner.value == 0 and resid.value == 0.0
    assert call(V=0, prec=3) == 0  # FEM_FP64_DF residuals
    w = lib.fem_pcg_refined_work_bytes(3, 1000, 300, 4)
    assert w >= lib.fem_pcg_work_bytes(3, 1000, 300, 1) + 4 * 1000 * 4 + 4 * 1000 * 8
    assert lib.fem_pcg_refined_work_bytes(4, 1000, 300, 4) == -1


def test_pcg_elasticity_validation(lib):
    """Argument checks of the elasticity solve, made before any CUDA call."""
    P, i64, cd, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    f = lib.fem_pcg_elasticity
    f.argtypes = [ci, i64, i64, P, P, P, P, ci, P, P, P, P, P, P, P, ci, cd, P, i64, P, P, ci, P]
    f.restype = ci
    lib.fem_pcg_elasticity_work_bytes.argtypes = [ci, i64, i64, ci]
    lib.fem_pcg_elasticity_work_bytes.restype = i64
    lib.fem_pcg_work_bytes.argtypes = [ci, i64, i64, ci]
    lib.fem_pcg_work_bytes.restype = i64
    fake = P(1 << 20)
    it, res = ctypes.c_int(-1), ctypes.c_double(-1.0)
    call = lambda V=0, prec=0, rtol=1e-8, mi=100: f(3, 0, V, fake, fake, fake, fake, 4, fake, fake, fake, fake, fake,
                                                  None, fake, mi, rtol, fake, 1 << 30, ctypes.byref(it),
                                                  ctypes.byref(res), prec, None)
    assert call(prec=7) == -1 and call(rtol=-1.0) == -1 and call(mi=-1) == -1
    assert call(V=0) == 0 and it.value == 0 and res.value == 0.0
    # three components per vertex: the vectors are three times the Laplacian solve's
    assert lib.fem_pcg_elasticity_work_bytes(3, 1000, 300, 0) > lib.fem_pcg_work_bytes(3, 1000, 300, 0)
    assert lib.fem_pcg_elasticity_work_bytes(4, 1000, 300, 0) == -1


def test_prepared_call_repeats_the_c_call_and_reports_its_status(lib):
    """A PreparedCall converts its arguments to ctypes values once and makes the same C
    call each time it is called; a failing status raises FemError every time (here the
    host-side check of dim, before any device work)."""
    from paper_1607_04245_gb300 import binding

    args = (4, 10, 10, None, None, None, None, 4, None, None, None, binding.FEM_FP32_MIXED, None)
    pc = binding.PreparedCall("fem_integrate_laplacian", args, keep=())
    assert all(isinstance(x, ctypes._SimpleCData) for x in pc._args)
    for _ in range(2):
        with pytest.raises(binding.FemError) as e:
            pc()
        assert e.value.status == -1 and "dim" in str(e.value)
