"""CPU FP64 oracle for P1 quadrature element integration -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. The product path (the CUDA library and its binding)
never does. The arithmetic lives in ``fem_oracle.c`` (plain C, FP64, one cell at a
time); this module compiles it with gcc and calls it through ctypes.

Functions take numpy arrays in the layouts documented in ``fem_oracle.c`` and
return new float64 arrays.
"""

from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fem_oracle.c")
_LIB = None


def lib_path() -> str:
    return os.path.join(_HERE, f"liboracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile fem_oracle.c into a shared library (OpenMP if the compiler has it)."""
    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", _SRC, "-lm"]
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    try:
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-o", tmp], capture_output=True, text=True)
        if r.returncode != 0:
            r = subprocess.run(base + ["-o", tmp], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"oracle build failed:\n{r.stderr}")
        os.replace(tmp, out)
    finally:
        if os.path.exists(tmp):
            os.unlink(tmp)
    return out


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        ci = ctypes.c_int
        lib.oracle_laplacian.argtypes = [ci, i64, i64, P, P, P, P, ci, P, P, P]
        lib.oracle_elasticity.argtypes = [ci, i64, i64, P, P, P, P, P, ci, P, P, P]
        lib.oracle_adjoint_laplacian.argtypes = [ci, i64, i64, P, P, P, P, ci, P, P, P, P, P]
        lib.oracle_reaction_diffusion.argtypes = [ci, i64, i64, P, P, P, P, ci, P, ctypes.c_double, ci, P, P, P]
        lib.oracle_pointwise.argtypes = [ci, P, ci, ci, ci, i64, i64, P, P, P, P, ci, P, P, P]
        for f in (lib.oracle_laplacian, lib.oracle_elasticity, lib.oracle_adjoint_laplacian,
                  lib.oracle_reaction_diffusion, lib.oracle_pointwise):
            f.restype = ci
        lib.oracle_num_threads.restype = ci
        lib.oracle_set_threads.argtypes = [ci]
        lib.oracle_set_threads.restype = None
        _LIB = lib
    return _LIB


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class OracleError(RuntimeError):
    pass


def _check(st):
    if st != 0:
        raise OracleError({-1: "bad argument", -5: "bad mesh"}.get(st, f"status {st}"))


def num_threads() -> int:
    return int(_lib().oracle_num_threads())


def set_threads(n: int) -> None:
    """Threads of the loops over cells (timing only; results do not depend on it)."""
    _lib().oracle_set_threads(int(n))


def laplacian(coords, conn, u, K, qpts, qw) -> np.ndarray:
    coords, u, K, qpts, qw = map(_f64, (coords, u, K, qpts, qw))
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    dim, V = coords.shape
    C = conn.shape[1]
    nq = qw.shape[0]
    out = np.zeros((dim + 1, C), dtype=np.float64)
    _check(_lib().oracle_laplacian(dim, C, V, _ptr(coords), _ptr(conn), _ptr(u), _ptr(K), nq,
                                   _ptr(qpts), _ptr(qw), _ptr(out)))
    return out


def elasticity(coords, conn, u, lam, mu, qpts, qw) -> np.ndarray:
    coords, u, lam, mu, qpts, qw = map(_f64, (coords, u, lam, mu, qpts, qw))
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    dim, V = coords.shape
    C = conn.shape[1]
    nq = qw.shape[0]
    out = np.zeros(((dim + 1) * dim, C), dtype=np.float64)
    _check(_lib().oracle_elasticity(dim, C, V, _ptr(coords), _ptr(conn), _ptr(u), _ptr(lam), _ptr(mu),
                                    nq, _ptr(qpts), _ptr(qw), _ptr(out)))
    return out


def adjoint_laplacian(coords, conn, u, K, qpts, qw, lam_adj):
    """Returns (dK [n_q][C], du [V]) for J = sum lambda . r."""
    coords, u, K, qpts, qw, lam_adj = map(_f64, (coords, u, K, qpts, qw, lam_adj))
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    dim, V = coords.shape
    C = conn.shape[1]
    nq = qw.shape[0]
    dK = np.zeros((nq, C), dtype=np.float64)
    du = np.zeros(V, dtype=np.float64)
    _check(_lib().oracle_adjoint_laplacian(dim, C, V, _ptr(coords), _ptr(conn), _ptr(u), _ptr(K), nq,
                                           _ptr(qpts), _ptr(qw), _ptr(lam_adj), _ptr(dK), _ptr(du)))
    return dK, du


def reaction_diffusion(coords, conn, u, a, a_space, c, qpts, qw, drift=0.0) -> np.ndarray:
    """Element vectors [dim+1][C] of f1 = a grad u, f0 = c u + drift grad a . grad u (a in
    P1: a_space=1, a[V]; in P0: a_space=0, a[C], grad a = 0; c [n_q][C] or None)."""
    coords, u, a, qpts, qw = map(_f64, (coords, u, a, qpts, qw))
    c = None if c is None else _f64(c)
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    dim, V = coords.shape
    C = conn.shape[1]
    nq = qw.shape[0]
    out = np.zeros((dim + 1, C), dtype=np.float64)
    _check(_lib().oracle_reaction_diffusion(dim, C, V, _ptr(coords), _ptr(conn), _ptr(u), _ptr(a), int(a_space),
                                            _ptr(c), float(drift), nq, _ptr(qpts), _ptr(qw), _ptr(out)))
    return out


POINTWISE_PHYSICS = {"laplacian": 0, "nonlinear": 1, "elasticity": 2, "reaction": 3}


def pointwise(physics, coords, conn, u, coef, qpts, qw, params=(0.0, 0.0, 0.0, 0.0)) -> np.ndarray:
    """Element vectors [(dim+1)*n_comp][C] of one of the oracle's pointwise physics
    (fem_oracle.c, oracle_pointwise): "laplacian" f1 = a0 grad u; "nonlinear" f1 =
    (p0 + p1 u + p2 u^2)(1 + p3 s(x)) grad u, s(x) = x_0 + 2 x_1 (+ 3 x_2); "elasticity" (Lame,
    a0 = lambda, a1 = mu);
    "reaction" f0 = a0 u + p0, f1 = a1 grad u. u is [V] or [n_comp][V], coef
    [n_coef][n_q][C] (or None)."""
    pid = POINTWISE_PHYSICS[physics]
    coords, qpts, qw = map(_f64, (coords, qpts, qw))
    u = _f64(u)
    if u.ndim == 1:
        u = u[None, :]
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    dim, V = coords.shape
    C = conn.shape[1]
    nq = qw.shape[0]
    n_comp = u.shape[0]
    coef = None if coef is None else _f64(coef)
    n_coef = 0 if coef is None else coef.shape[0]
    if coef is not None and coef.shape != (n_coef, nq, C):
        raise ValueError("coef must be [n_coef][n_q][C]")
    p = _f64(np.asarray(params, dtype=np.float64).reshape(-1)[:4])
    out = np.zeros(((dim + 1) * n_comp, C), dtype=np.float64)
    _check(_lib().oracle_pointwise(pid, _ptr(p), dim, n_comp, n_coef, C, V, _ptr(coords), _ptr(conn), _ptr(u),
                                   _ptr(coef), nq, _ptr(qpts), _ptr(qw), _ptr(out)))
    return out


# convenience wrappers over a workloads.Case (the oracle does not import workloads;
# it reads the attributes by name)
def residual_for(case) -> np.ndarray:
    m, r = case.mesh, case.rule
    if case.physics == "laplacian":
        return laplacian(m.coords, m.conn, case.u, case.K, r.points, r.weights)
    return elasticity(m.coords, m.conn, case.u, case.lam, case.mu, r.points, r.weights)


def adjoint_for(case, lam_adj=None):
    m, r = case.mesh, case.rule
    return adjoint_laplacian(m.coords, m.conn, case.u, case.K, r.points, r.weights,
                             case.adj if lam_adj is None else lam_adj)
