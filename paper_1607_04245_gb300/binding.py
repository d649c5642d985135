"""Thin Python binding of libfem's C ABI (include/fem.h).

Every function here has the name of the C entry point it calls and does argument
marshalling only: it checks tensor devices, dtypes, shapes and contiguity, derives
the sizes, allocates outputs with torch when the caller passes none, and hands raw
pointers and the current CUDA stream to the library. All arithmetic runs in the
library's CUDA kernels. There is no fallback: if libfem.so is missing or the call
fails, a RuntimeError is raised.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple, Union

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfem.so")

FEM_FP64, FEM_FP32_MIXED, FEM_FP32, FEM_FP64_DF = 0, 1, 2, 3
_PREC_NAMES = {"fp64": FEM_FP64, "mixed": FEM_FP32_MIXED, "fp32_mixed": FEM_FP32_MIXED, "fp32": FEM_FP32,
               "fp64_df": FEM_FP64_DF}
FEM_MAX_QPTS = 32

_lib = None


class FemError(RuntimeError):
    def __init__(self, fn: str, status: int, message: str):
        super().__init__(f"{fn} failed with status {status}: {message}")
        self.status = status


def lib():
    """The loaded libfem (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfem.so not found at {LIB_PATH}: build it with __graft_entry__.build() "
                               "or python -m paper_1607_04245_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        P, i64, ci, cd = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        sig = {
            "fem_integrate_laplacian": [ci, i64, i64, P, P, P, P, ci, P, P, P, ci, P],
            "fem_integrate_laplacian_fields": [ci, i64, i64, P, P, ci, P, P, ci, P, P, P, ci, P],
            "fem_integrate_elasticity": [ci, i64, i64, P, P, P, P, P, ci, P, P, P, ci, P],
            "fem_adjoint_laplacian": [ci, i64, i64, P, P, P, P, ci, P, P, P, P, P, P, P, P, ci, P],
            "fem_build_node2cell": [ci, i64, i64, P, P, P, P, P],
            "fem_gather_nodes": [ci, ci, i64, i64, P, P, P, P, ci, P],
            "fem_check_mesh": [ci, i64, i64, P, P, P, P],
            "fem_probe": [ci, i64, ci, P, P],
            "fem_set_mixed_threshold": [cd],
            "fem_device_error": [P],
            "fem_precompute_geometry": [ci, i64, i64, P, P, P, ci, P],
            "fem_integrate_reaction_diffusion": [ci, i64, i64, P, P, P, P, ci, P, cd, ci, P, P, P, ci, P],
            "fem_element_values": [ci, i64, i64, P, P, P, ci, P],
            "fem_integrate_laplacian_host": [ci, i64, i64, P, P, P, P, ci, P, P, P, P, i64, ci, ci, P],
            "fem_integrate_laplacian_transposed": [ci, i64, P, P, ci, P, P, P, P, ci, ci, ci, P],
            "fem_pcg_laplacian": [ci, i64, i64, P, P, P, ci, P, P, P, P, P, P, P, ci, cd, P, i64, P, P, ci, P],
            "fem_pcg_elasticity": [ci, i64, i64, P, P, P, P, ci, P, P, P, P, P, P, P, ci, cd, P, i64, P, P, ci, P],
            "fem_pcg_elasticity_refined": [ci, i64, i64, P, P, P, P, ci, P, P, P, P, P, P, P, ci, ci, cd, cd, P, i64,
                                           P, P, P, ci, P],
            "fem_pcg_laplacian_refined": [ci, i64, i64, P, P, P, ci, P, P, P, P, P, P, P, ci, ci, cd, cd, P, i64, P,
                                          P, P, ci, P],
            "fem_integrate_laplacian_geom": [ci, i64, i64, P, P, P, ci, P, P, P, P, ci, P],
            "fem_selftest_wait": [i64, P],
            "fem_selftest_quotient": [i64, P, P, P, P, P],
            "fem_prepare_vertices": [ci, i64, P, P, P],
            "fem_integrate_laplacian_prepared": [ci, i64, i64, P, P, P, P, P, ci, P, P, P, P],
            "fem_integrate_pointwise": [ctypes.c_char_p, ctypes.c_char_p, ci, ci, ci, i64, i64, P, P, P, P, ci, P,
                                        P, P, ci, P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ci
        L.fem_get_mixed_threshold.argtypes = []
        L.fem_get_mixed_threshold.restype = cd
        L.fem_host_work_bytes.argtypes = [ci, i64, i64, ci, ci, ci]
        L.fem_host_work_bytes.restype = i64
        L.fem_pcg_work_bytes.argtypes = [ci, i64, i64, ci]
        L.fem_pcg_work_bytes.restype = i64
        L.fem_pcg_elasticity_work_bytes.argtypes = [ci, i64, i64, ci]
        L.fem_pcg_elasticity_work_bytes.restype = i64
        L.fem_pcg_elasticity_refined_work_bytes.argtypes = [ci, i64, i64, ci]
        L.fem_pcg_elasticity_refined_work_bytes.restype = i64
        L.fem_pcg_refined_work_bytes.argtypes = [ci, i64, i64, ci]
        L.fem_pcg_refined_work_bytes.restype = i64
        L.fem_prepared_record_floats.argtypes = [ci]
        L.fem_prepared_record_floats.restype = i64
        L.fem_node2cell_work_size.argtypes = [i64]
        L.fem_node2cell_work_size.restype = i64
        for name in ("fem_last_error", "fem_version"):
            getattr(L, name).restype = ctypes.c_char_p
        L.fem_status_string.argtypes = [ci]
        L.fem_status_string.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(fn: str, st: int):
    if st != 0:
        raise FemError(fn, st, lib().fem_last_error().decode())


def precision(p: Union[int, str]) -> int:
    if isinstance(p, str):
        return _PREC_NAMES[p.lower()]
    if p not in (FEM_FP64, FEM_FP32_MIXED, FEM_FP32, FEM_FP64_DF):
        raise ValueError(f"unknown precision {p}")
    return int(p)


def value_dtype(prec) -> torch.dtype:
    return torch.float64 if precision(prec) in (FEM_FP64, FEM_FP64_DF) else torch.float32


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _dev(t: Optional[torch.Tensor], name: str, dtype: torch.dtype, shape=None, device=None) -> int:
    if t is None:
        raise ValueError(f"{name} is required")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr() if t.numel() else 0


class _HostTable:
    """A float64 host table kept alive for the duration of a call."""

    def __init__(self, a, shape=None, name="table"):
        if a is None:
            self.arr, self.ptr = None, None
            return
        if isinstance(a, torch.Tensor):
            a = a.detach().cpu().numpy()
        self.arr = np.ascontiguousarray(a, dtype=np.float64)
        if shape is not None and self.arr.shape != tuple(shape):
            raise ValueError(f"{name} has shape {self.arr.shape}, expected {tuple(shape)}")
        self.ptr = self.arr.ctypes.data


def _mesh_sizes(coords: torch.Tensor, conn: torch.Tensor):
    if coords.dim() != 2 or conn.dim() != 2:
        raise ValueError("coords must be (dim, V) and conn (dim+1, C)")
    dim, V = coords.shape
    if conn.shape[0] != dim + 1:
        raise ValueError(f"conn must have dim+1 = {dim + 1} rows")
    return int(dim), int(V), int(conn.shape[1])


class PreparedCall:
    """One C-ABI call whose arguments were validated and marshalled once, for loops that
    repeat it on the same buffers (Python's per-call checks cost about as much host time
    as a small kernel takes on the device). Calling it runs the plain entry point again
    with the same pointers, sizes and stream; the tensors and host tables it was made from
    stay referenced for its life and must keep their storage. prepared_integrate_laplacian
    and prepared_integrate_elasticity make one; so do fem_integrate_laplacian_fields,
    fem_integrate_laplacian_prepared, fem_integrate_pointwise,
    fem_integrate_reaction_diffusion, fem_integrate_laplacian_geom and
    fem_adjoint_laplacian when given prepare=True (they then run nothing)."""

    def __init__(self, name: str, args, keep):
        self._f = getattr(lib(), name)
        self._name = name
        self._args = tuple(t(a) for t, a in zip(self._f.argtypes, args))  # converted once
        self._keep = keep

    def __call__(self):
        st = self._f(*self._args)
        if st != 0:
            _check(self._name, st)


def _run(name: str, args, keep, prepare: bool):
    """Call entry point `name` with marshalled `args`, or return that call as a
    PreparedCall (prepare=True) without running it."""
    if prepare:
        return PreparedCall(name, args, keep)
    _check(name, getattr(lib(), name)(*args))
    return None


def _laplacian_call(coords, conn, u, K, qpts, qw, out, prec, stream):
    p = precision(prec)
    dt = value_dtype(p)
    dim, V, C = _mesh_sizes(coords, conn)
    nq = int(np.asarray(qw).shape[0]) if not isinstance(qw, torch.Tensor) else int(qw.shape[0])
    dev = coords.device
    if out is None:
        out = torch.empty((dim + 1, C), dtype=dt, device=dev)
    qp, w = _HostTable(qpts, (nq, dim), "qpts"), _HostTable(qw, (nq,), "qw")
    args = (dim, C, V, _dev(coords, "coords", torch.float64, device=dev), _dev(conn, "conn", torch.int32, device=dev),
            _dev(u, "u", dt, (V,), dev), _dev(K, "K", dt, (nq, C), dev), nq, qp.ptr, w.ptr,
            _dev(out, "out", dt, (dim + 1, C), dev), p, _stream(stream))
    return out, args, (coords, conn, u, K, out, qp, w)


def fem_integrate_laplacian(coords, conn, u, K, qpts, qw, out=None, prec="mixed", stream=None) -> torch.Tensor:
    """Element residuals [dim+1][C] of the variable-coefficient Laplacian."""
    out, args, _keep = _laplacian_call(coords, conn, u, K, qpts, qw, out, prec, stream)
    _check("fem_integrate_laplacian", lib().fem_integrate_laplacian(*args))
    return out


def prepared_integrate_laplacian(coords, conn, u, K, qpts, qw, out, prec="mixed", stream=None) -> PreparedCall:
    """fem_integrate_laplacian on fixed buffers as a PreparedCall: each call of the result
    launches the residual into `out` again."""
    _, args, keep = _laplacian_call(coords, conn, u, K, qpts, qw, out, prec, stream)
    return PreparedCall("fem_integrate_laplacian", args, keep)


def fem_integrate_laplacian_fields(coords, conn, u, K, qpts, qw, out=None, prec="mixed", stream=None, prepare=False):
    """Element residuals [F][dim+1][C] of the variable-coefficient Laplacian for F nodal
    fields u [F][V] on one mesh (geometry computed once per cell)."""
    p = precision(prec)
    dt = value_dtype(p)
    dim, V, C = _mesh_sizes(coords, conn)
    nf = int(u.shape[0])
    nq = int(np.asarray(qw).shape[0]) if not isinstance(qw, torch.Tensor) else int(qw.shape[0])
    dev = coords.device
    if out is None:
        out = torch.empty((nf, dim + 1, C), dtype=dt, device=dev)
    qp, w = _HostTable(qpts, (nq, dim), "qpts"), _HostTable(qw, (nq,), "qw")
    args = (
        dim, C, V, _dev(coords, "coords", torch.float64, device=dev), _dev(conn, "conn", torch.int32, device=dev), nf,
        _dev(u, "u", dt, (nf, V), dev), _dev(K, "K", dt, (nq, C), dev), nq, qp.ptr, w.ptr,
        _dev(out, "out", dt, (nf, dim + 1, C), dev), p, _stream(stream))
    pc = _run("fem_integrate_laplacian_fields", args, (coords, conn, u, K, out, qp, w), prepare)
    if prepare:
        return pc
    return out


def _elasticity_call(coords, conn, u, lam, mu, qpts, qw, out, prec, stream):
    p = precision(prec)
    dt = value_dtype(p)
    dim, V, C = _mesh_sizes(coords, conn)
    nq = int(np.asarray(qw).shape[0]) if not isinstance(qw, torch.Tensor) else int(qw.shape[0])
    dev = coords.device
    if out is None:
        out = torch.empty(((dim + 1) * dim, C), dtype=dt, device=dev)
    qp, w = _HostTable(qpts, (nq, dim), "qpts"), _HostTable(qw, (nq,), "qw")
    args = (dim, C, V, _dev(coords, "coords", torch.float64, device=dev), _dev(conn, "conn", torch.int32, device=dev),
            _dev(u, "u", dt, (dim, V), dev), _dev(lam, "lam", dt, (nq, C), dev), _dev(mu, "mu", dt, (nq, C), dev),
            nq, qp.ptr, w.ptr, _dev(out, "out", dt, ((dim + 1) * dim, C), dev), p, _stream(stream))
    return out, args, (coords, conn, u, lam, mu, out, qp, w)


def fem_integrate_elasticity(coords, conn, u, lam, mu, qpts, qw, out=None, prec="mixed", stream=None) -> torch.Tensor:
    """Element residuals [(dim+1)*dim][C] of linear elasticity (row b*dim + k)."""
    out, args, _keep = _elasticity_call(coords, conn, u, lam, mu, qpts, qw, out, prec, stream)
    _check("fem_integrate_elasticity", lib().fem_integrate_elasticity(*args))
    return out


def prepared_integrate_elasticity(coords, conn, u, lam, mu, qpts, qw, out, prec="mixed",
                                  stream=None) -> PreparedCall:
    """fem_integrate_elasticity on fixed buffers as a PreparedCall."""
    _, args, keep = _elasticity_call(coords, conn, u, lam, mu, qpts, qw, out, prec, stream)
    return PreparedCall("fem_integrate_elasticity", args, keep)


def fem_prepare_vertices(coords, rec=None, stream=None) -> torch.Tensor:
    """Per-mesh vertex records [V][8] (3D) or [V][4] (2D), float32: each coordinate's
    (hi, lo) split, for fem_integrate_laplacian_prepared."""
    dim, V = int(coords.shape[0]), int(coords.shape[1])
    R = int(lib().fem_prepared_record_floats(dim))
    if R < 0:
        raise ValueError("coords must be (2, V) or (3, V)")
    dev = coords.device
    rec = torch.empty((V, R), dtype=torch.float32, device=dev) if rec is None else rec
    _check("fem_prepare_vertices", lib().fem_prepare_vertices(
        dim, V, _dev(coords, "coords", torch.float64, device=dev), _dev(rec, "rec", torch.float32, (V, R), dev),
        _stream(stream)))
    return rec


def fem_integrate_laplacian_prepared(coords, rec, conn, u, K, qpts, qw, out=None, stream=None, prepare=False):
    """fem_integrate_laplacian (FP32-mixed) from the prepared vertex records: bitwise the same
    element vectors [dim+1][C]."""
    dim, V, C = _mesh_sizes(coords, conn)
    nq = int(np.asarray(qw).shape[0]) if not isinstance(qw, torch.Tensor) else int(qw.shape[0])
    dev = coords.device
    R = int(lib().fem_prepared_record_floats(dim))
    if out is None:
        out = torch.empty((dim + 1, C), dtype=torch.float32, device=dev)
    qp, w = _HostTable(qpts, (nq, dim), "qpts"), _HostTable(qw, (nq,), "qw")
    args = (
        dim, C, V, _dev(coords, "coords", torch.float64, device=dev), _dev(rec, "rec", torch.float32, (V, R), dev),
        _dev(conn, "conn", torch.int32, device=dev), _dev(u, "u", torch.float32, (V,), dev),
        _dev(K, "K", torch.float32, (nq, C), dev), nq, qp.ptr, w.ptr,
        _dev(out, "out", torch.float32, (dim + 1, C), dev), _stream(stream))
    pc = _run("fem_integrate_laplacian_prepared", args, (coords, rec, conn, u, K, out, qp, w), prepare)
    if prepare:
        return pc
    return out


def fem_integrate_pointwise(coords, conn, u, coef, qpts, qw, f1=None, f0=None, out=None, prec="mixed",
                            stream=None, prepare=False):
    """Element vectors [(dim+1)*n_comp][C] of Eq. 2 for pointwise functions given as CUDA
    source text: f1 and f0 are function bodies (see fem_integrate_pointwise in
    include/fem.h for the names in scope), compiled at run time and cached. u is [V] or
    [n_comp][V]; coef is [n_coef][n_q][C] or None. An empty mesh (C = 0) only compiles."""
    p = precision(prec)
    dt = value_dtype(p)
    dim, V, C = _mesh_sizes(coords, conn)
    nq = int(np.asarray(qw).shape[0]) if not isinstance(qw, torch.Tensor) else int(qw.shape[0])
    dev = coords.device
    n_comp = 1 if u.dim() == 1 else int(u.shape[0])
    n_coef = 0 if coef is None else int(coef.shape[0])
    if out is None:
        out = torch.empty(((dim + 1) * n_comp, C), dtype=dt, device=dev)
    qp, w = _HostTable(qpts, (nq, dim), "qpts"), _HostTable(qw, (nq,), "qw")
    enc = lambda t: None if t is None else t.encode()
    args = (
        enc(f0), enc(f1), dim, n_comp, n_coef, C, V, _dev(coords, "coords", torch.float64, device=dev),
        _dev(conn, "conn", torch.int32, device=dev),
        _dev(u, "u", dt, (V,) if u.dim() == 1 else (n_comp, V), dev),
        None if coef is None else _dev(coef, "coef", dt, (n_coef, nq, C), dev), nq, qp.ptr, w.ptr,
        _dev(out, "out", dt, ((dim + 1) * n_comp, C), dev), p, _stream(stream))
    pc = _run("fem_integrate_pointwise", args, (coords, conn, u, coef, out, qp, w), prepare)
    if prepare:
        return pc
    return out


def fem_integrate_reaction_diffusion(coords, conn, u, a, qpts, qw, c=None, a_space=1, drift=0.0, out=None,
                                     prec="mixed", stream=None, prepare=False):
    """Element vectors [dim+1][C] of f1 = a grad u, f0 = c u + drift grad a . grad u (Eqs. 2
    and 8): a is P1 nodal ([V], a_space=1) or P0 ([C], a_space=0, grad a = 0); c is
    [n_q][C] or None."""
    p = precision(prec)
    dt = value_dtype(p)
    dim, V, C = _mesh_sizes(coords, conn)
    nq = int(np.asarray(qw).shape[0]) if not isinstance(qw, torch.Tensor) else int(qw.shape[0])
    dev = coords.device
    if qpts is None:
        raise ValueError("qpts is required")
    out = torch.empty((dim + 1, C), dtype=dt, device=dev) if out is None else out
    qp, w = _HostTable(qpts, (nq, dim), "qpts"), _HostTable(qw, (nq,), "qw")
    args = (
        dim, C, V, _dev(coords, "coords", torch.float64, device=dev), _dev(conn, "conn", torch.int32, device=dev),
        _dev(u, "u", dt, (V,), dev), _dev(a, "a", dt, (V,) if a_space == 1 else (C,), dev), int(a_space),
        None if c is None else _dev(c, "c", dt, (nq, C), dev), float(drift), nq, qp.ptr, w.ptr,
        _dev(out, "out", dt, (dim + 1, C), dev), p, _stream(stream))
    pc = _run("fem_integrate_reaction_diffusion", args, (coords, conn, u, a, c, out, qp, w), prepare)
    if prepare:
        return pc
    return out


def fem_pcg_laplacian(coords, conn, K, qpts, qw, node_ptr, node_idx, fixed, x, b=None, max_iter=1000, rtol=1e-8,
                      work=None, prec="fp64", stream=None):
    """Solve the assembled Laplacian system on the free vertices (Dirichlet values in x).
    Returns (x, iterations, relative residual)."""
    p = precision(prec)
    dt = value_dtype(p)
    dim, V, C = _mesh_sizes(coords, conn)
    nq = int(np.asarray(qw).shape[0]) if not isinstance(qw, torch.Tensor) else int(qw.shape[0])
    dev = coords.device
    need = int(lib().fem_pcg_work_bytes(dim, C, V, p))
    if work is None:
        work = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    qp, w = _HostTable(qpts, (nq, dim), "qpts"), _HostTable(qw, (nq,), "qw")
    iters, resid = ctypes.c_int(0), ctypes.c_double(0.0)
    st = lib().fem_pcg_laplacian(
        dim, C, V, _dev(coords, "coords", torch.float64, device=dev), _dev(conn, "conn", torch.int32, device=dev),
        _dev(K, "K", dt, (nq, C), dev), nq, qp.ptr, w.ptr, _dev(node_ptr, "node_ptr", torch.int32, (V + 1,), dev),
        _dev(node_idx, "node_idx", torch.int32, ((dim + 1) * C,), dev), _dev(fixed, "fixed", torch.uint8, (V,), dev),
        None if b is None else _dev(b, "b", dt, (V,), dev), _dev(x, "x", dt, (V,), dev), int(max_iter), float(rtol),
        _dev(work, "work", torch.uint8, None, dev), int(work.numel()), ctypes.byref(iters), ctypes.byref(resid), p,
        _stream(stream))
    _check("fem_pcg_laplacian", st)
    return x, int(iters.value), float(resid.value)


def fem_pcg_elasticity(coords, conn, lam, mu, qpts, qw, node_ptr, node_idx, fixed, x, b=None, max_iter=1000,
                       rtol=1e-8, work=None, prec="fp64", stream=None):
    """Solve the assembled linear-elasticity system (x, b: [dim][V]) on the free vertices
    (Dirichlet values of all components in x). Returns (x, iterations, relative residual)."""
    p = precision(prec)
    dt = value_dtype(p)
    dim, V, C = _mesh_sizes(coords, conn)
    nq = int(np.asarray(qw).shape[0]) if not isinstance(qw, torch.Tensor) else int(qw.shape[0])
    dev = coords.device
    need = int(lib().fem_pcg_elasticity_work_bytes(dim, C, V, p))
    if work is None:
        work = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    qp, w = _HostTable(qpts, (nq, dim), "qpts"), _HostTable(qw, (nq,), "qw")
    iters, resid = ctypes.c_int(0), ctypes.c_double(0.0)
    st = lib().fem_pcg_elasticity(
        dim, C, V, _dev(coords, "coords", torch.float64, device=dev), _dev(conn, "conn", torch.int32, device=dev),
        _dev(lam, "lam", dt, (nq, C), dev), _dev(mu, "mu", dt, (nq, C), dev), nq, qp.ptr, w.ptr,
        _dev(node_ptr, "node_ptr", torch.int32, (V + 1,), dev),
        _dev(node_idx, "node_idx", torch.int32, ((dim + 1) * C,), dev), _dev(fixed, "fixed", torch.uint8, (V,), dev),
        None if b is None else _dev(b, "b", dt, (dim, V), dev), _dev(x, "x", dt, (dim, V), dev), int(max_iter),
        float(rtol), _dev(work, "work", torch.uint8, None, dev), int(work.numel()), ctypes.byref(iters),
        ctypes.byref(resid), p, _stream(stream))
    _check("fem_pcg_elasticity", st)
    return x, int(iters.value), float(resid.value)


def fem_pcg_laplacian_refined(coords, conn, K, qpts, qw, node_ptr, node_idx, fixed, x, b=None, max_outer=20,
                              max_inner=2000, inner_rtol=1e-4, rtol=1e-8, work=None, residual_prec="fp64",
                              stream=None):
    """Mixed-precision iterative refinement of the assembled Laplacian solve: float64 x, b
    and K; corrections by the FP32-mixed PCG, true residuals in residual_prec ("fp64" or
    "fp64_df"). Returns (x, outer steps, float32 PCG iterations, relative residual)."""
    dim, V, C = _mesh_sizes(coords, conn)
    nq = int(np.asarray(qw).shape[0]) if not isinstance(qw, torch.Tensor) else int(qw.shape[0])
    dev = coords.device
    need = int(lib().fem_pcg_refined_work_bytes(dim, C, V, nq))
    if need < 0:
        raise ValueError("bad sizes")
    if work is None:
        work = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    qp, w = _HostTable(qpts, (nq, dim), "qpts"), _HostTable(qw, (nq,), "qw")
    outer, inner, resid = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    f64 = torch.float64
    st = lib().fem_pcg_laplacian_refined(
        dim, C, V, _dev(coords, "coords", f64, device=dev), _dev(conn, "conn", torch.int32, device=dev),
        _dev(K, "K", f64, (nq, C), dev), nq, qp.ptr, w.ptr, _dev(node_ptr, "node_ptr", torch.int32, (V + 1,), dev),
        _dev(node_idx, "node_idx", torch.int32, ((dim + 1) * C,), dev), _dev(fixed, "fixed", torch.uint8, (V,), dev),
        None if b is None else _dev(b, "b", f64, (V,), dev), _dev(x, "x", f64, (V,), dev), int(max_outer),
        int(max_inner), float(inner_rtol), float(rtol), _dev(work, "work", torch.uint8, None, dev), int(work.numel()),
        ctypes.byref(outer), ctypes.byref(inner), ctypes.byref(resid), precision(residual_prec), _stream(stream))
    _check("fem_pcg_laplacian_refined", st)
    return x, int(outer.value), int(inner.value), float(resid.value)


def fem_pcg_elasticity_refined(coords, conn, lam, mu, qpts, qw, node_ptr, node_idx, fixed, x, b=None, max_outer=20,
                               max_inner=5000, inner_rtol=1e-4, rtol=1e-8, work=None, residual_prec="fp64",
                               stream=None):
    """Mixed-precision iterative refinement of the assembled elasticity solve (float64
    lam, mu, b, x [dim][V]). Returns (x, outer steps, float32 PCG iterations, relative residual)."""
    dim, V, C = _mesh_sizes(coords, conn)
    nq = int(np.asarray(qw).shape[0]) if not isinstance(qw, torch.Tensor) else int(qw.shape[0])
    dev = coords.device
    need = int(lib().fem_pcg_elasticity_refined_work_bytes(dim, C, V, nq))
    if need < 0:
        raise ValueError("bad sizes")
    if work is None:
        work = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    qp, w = _HostTable(qpts, (nq, dim), "qpts"), _HostTable(qw, (nq,), "qw")
    outer, inner, resid = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    f64 = torch.float64
    st = lib().fem_pcg_elasticity_refined(
        dim, C, V, _dev(coords, "coords", f64, device=dev), _dev(conn, "conn", torch.int32, device=dev),
        _dev(lam, "lam", f64, (nq, C), dev), _dev(mu, "mu", f64, (nq, C), dev), nq, qp.ptr, w.ptr,
        _dev(node_ptr, "node_ptr", torch.int32, (V + 1,), dev),
        _dev(node_idx, "node_idx", torch.int32, ((dim + 1) * C,), dev), _dev(fixed, "fixed", torch.uint8, (V,), dev),
        None if b is None else _dev(b, "b", f64, (dim, V), dev), _dev(x, "x", f64, (dim, V), dev), int(max_outer),
        int(max_inner), float(inner_rtol), float(rtol), _dev(work, "work", torch.uint8, None, dev), int(work.numel()),
        ctypes.byref(outer), ctypes.byref(inner), ctypes.byref(resid), precision(residual_prec), _stream(stream))
    _check("fem_pcg_elasticity_refined", st)
    return x, int(outer.value), int(inner.value), float(resid.value)


def _host(t: torch.Tensor, name: str, dtype: torch.dtype, shape) -> int:
    if t.is_cuda:
        raise ValueError(f"{name} must be a host tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr() if t.numel() else 0


def fem_integrate_laplacian_host(coords_h, conn_h, u_h, K_h, qpts, qw, out_h, work, chunks=4, prec="mixed",
                                 stream=None) -> torch.Tensor:
    """Laplacian element residuals from host tensors (pinned for overlap) into out_h; `work`
    is a device uint8 tensor of at least fem_host_work_bytes() bytes. Results are valid
    once `stream` has completed."""
    p = precision(prec)
    dt = value_dtype(p)
    dim, V = int(coords_h.shape[0]), int(coords_h.shape[1])
    C = int(conn_h.shape[1])
    nq = int(np.asarray(qw).shape[0]) if not isinstance(qw, torch.Tensor) else int(qw.shape[0])
    qp, w = _HostTable(qpts, (nq, dim), "qpts"), _HostTable(qw, (nq,), "qw")
    st = lib().fem_integrate_laplacian_host(
        dim, C, V, _host(coords_h, "coords_h", torch.float64, (dim, V)), _host(conn_h, "conn_h", torch.int32,
                                                                              (dim + 1, C)),
        _host(u_h, "u_h", dt, (V,)), _host(K_h, "K_h", dt, (nq, C)), nq, qp.ptr, w.ptr,
        _host(out_h, "out_h", dt, (dim + 1, C)), _dev(work, "work", torch.uint8, None), int(work.numel()),
        int(chunks), p, _stream(stream))
    _check("fem_integrate_laplacian_host", st)
    return out_h


def fem_host_work_bytes(dim: int, n_cells: int, n_verts: int, n_q: int, prec="mixed", chunks: int = 4) -> int:
    return int(lib().fem_host_work_bytes(dim, n_cells, n_verts, n_q, precision(prec), chunks))


def fem_element_values(conn, n_verts: int, u, ue=None, prec="mixed", stream=None) -> torch.Tensor:
    """Element basis coefficients ue[b][e] = u[conn[b][e]]."""
    p = precision(prec)
    dt = value_dtype(p)
    dim, C = int(conn.shape[0]) - 1, int(conn.shape[1])
    dev = conn.device
    ue = torch.empty((dim + 1, C), dtype=dt, device=dev) if ue is None else ue
    st = lib().fem_element_values(dim, C, int(n_verts), _dev(conn, "conn", torch.int32, device=dev),
                                  _dev(u, "u", dt, (n_verts,), dev), _dev(ue, "ue", dt, (dim + 1, C), dev), p,
                                  _stream(stream))
    _check("fem_element_values", st)
    return ue


def fem_integrate_laplacian_transposed(ue, K, qpts, qw, geom, cells_per_batch=64, batches_per_block=4, out=None,
                                       prec="mixed", stream=None) -> torch.Tensor:
    """The paper's thread-transposition kernel: element residuals [dim+1][C]."""
    p = precision(prec)
    dt = value_dtype(p)
    dim, C = int(ue.shape[0]) - 1, int(ue.shape[1])
    nq = int(np.asarray(qw).shape[0]) if not isinstance(qw, torch.Tensor) else int(qw.shape[0])
    dev = ue.device
    out = torch.empty((dim + 1, C), dtype=dt, device=dev) if out is None else out
    qp, w = _HostTable(qpts, (nq, dim), "qpts"), _HostTable(qw, (nq,), "qw")
    st = lib().fem_integrate_laplacian_transposed(
        dim, C, _dev(ue, "ue", dt, (dim + 1, C), dev), _dev(K, "K", dt, (nq, C), dev), nq, qp.ptr, w.ptr,
        _dev(geom, "geom", dt, (dim * dim + 1, C), dev), _dev(out, "out", dt, (dim + 1, C), dev),
        int(cells_per_batch), int(batches_per_block), p, _stream(stream))
    _check("fem_integrate_laplacian_transposed", st)
    return out


def fem_precompute_geometry(coords, conn, geom=None, prec="mixed", stream=None) -> torch.Tensor:
    """Per-cell geometry [dim*dim + 1][C]: J^{-1} rows (row-major) then det J."""
    p = precision(prec)
    dt = value_dtype(p)
    dim, V, C = _mesh_sizes(coords, conn)
    dev = coords.device
    geom = torch.empty((dim * dim + 1, C), dtype=dt, device=dev) if geom is None else geom
    st = lib().fem_precompute_geometry(dim, C, V, _dev(coords, "coords", torch.float64, device=dev),
                                       _dev(conn, "conn", torch.int32, device=dev),
                                       _dev(geom, "geom", dt, (dim * dim + 1, C), dev), p, _stream(stream))
    _check("fem_precompute_geometry", st)
    return geom


def fem_integrate_laplacian_geom(conn, n_verts: int, u, K, qpts, qw, geom, out=None, prec="mixed",
                                 stream=None, prepare=False):
    """Laplacian element residuals [dim+1][C] from the precomputed geometry."""
    p = precision(prec)
    dt = value_dtype(p)
    dim, C = int(conn.shape[0]) - 1, int(conn.shape[1])
    nq = int(np.asarray(qw).shape[0]) if not isinstance(qw, torch.Tensor) else int(qw.shape[0])
    dev = conn.device
    out = torch.empty((dim + 1, C), dtype=dt, device=dev) if out is None else out
    qp, w = _HostTable(qpts, (nq, dim), "qpts"), _HostTable(qw, (nq,), "qw")
    args = (
        dim, C, int(n_verts), _dev(conn, "conn", torch.int32, device=dev), _dev(u, "u", dt, (n_verts,), dev),
        _dev(K, "K", dt, (nq, C), dev), nq, qp.ptr, w.ptr, _dev(geom, "geom", dt, (dim * dim + 1, C), dev),
        _dev(out, "out", dt, (dim + 1, C), dev), p, _stream(stream))
    pc = _run("fem_integrate_laplacian_geom", args, (conn, u, K, geom, out, qp, w), prepare)
    if prepare:
        return pc
    return out


def fem_build_node2cell(conn, n_verts: int, node_ptr=None, node_idx=None, work=None, stream=None):
    """Vertex-to-(cell, local vertex) lists: (node_ptr [V+1], node_idx [(dim+1)*C])."""
    dim = int(conn.shape[0]) - 1
    C = int(conn.shape[1])
    dev = conn.device
    if node_ptr is None:
        node_ptr = torch.empty(n_verts + 1, dtype=torch.int32, device=dev)
    if node_idx is None:
        node_idx = torch.empty((dim + 1) * C, dtype=torch.int32, device=dev)
    if work is None:
        work = torch.empty(max(1, lib().fem_node2cell_work_size(n_verts)), dtype=torch.int32, device=dev)
    if work.numel() < lib().fem_node2cell_work_size(n_verts):
        raise ValueError("work is too small")
    st = lib().fem_build_node2cell(dim, C, n_verts, _dev(conn, "conn", torch.int32, device=dev),
                                   _dev(node_ptr, "node_ptr", torch.int32, (n_verts + 1,), dev),
                                   _dev(node_idx, "node_idx", torch.int32, ((dim + 1) * C,), dev),
                                   _dev(work, "work", torch.int32, None, dev), _stream(stream))
    _check("fem_build_node2cell", st)
    return node_ptr, node_idx


def fem_adjoint_laplacian(coords, conn, u, K, qpts, qw, lam_adj, node_ptr, node_idx, dK=None, du=None,
                          scratch=None, prec="mixed", stream=None, prepare=False):
    """Gradient of J = sum lambda . r: returns (dK [n_q][C], du [V])."""
    p = precision(prec)
    dt = value_dtype(p)
    dim, V, C = _mesh_sizes(coords, conn)
    nq = int(np.asarray(qw).shape[0]) if not isinstance(qw, torch.Tensor) else int(qw.shape[0])
    dev = coords.device
    dK = torch.empty((nq, C), dtype=dt, device=dev) if dK is None else dK
    du = torch.empty(V, dtype=dt, device=dev) if du is None else du
    scratch = torch.empty((dim + 1, C), dtype=dt, device=dev) if scratch is None else scratch
    qp, w = _HostTable(qpts, (nq, dim), "qpts"), _HostTable(qw, (nq,), "qw")
    args = (
        dim, C, V, _dev(coords, "coords", torch.float64, device=dev), _dev(conn, "conn", torch.int32, device=dev),
        _dev(u, "u", dt, (V,), dev), _dev(K, "K", dt, (nq, C), dev), nq, qp.ptr, w.ptr,
        _dev(lam_adj, "lambda", dt, (dim + 1, C), dev), _dev(dK, "dK", dt, (nq, C), dev),
        _dev(du, "du", dt, (V,), dev), _dev(node_ptr, "node_ptr", torch.int32, (V + 1,), dev),
        _dev(node_idx, "node_idx", torch.int32, ((dim + 1) * C,), dev),
        _dev(scratch, "scratch", dt, (dim + 1, C), dev), p, _stream(stream))
    pc = _run("fem_adjoint_laplacian", args, (coords, conn, u, K, lam_adj, node_ptr, node_idx, dK, du, scratch, qp, w), prepare)
    if prepare:
        return pc
    return dK, du


def fem_gather_nodes(elem, node_ptr, node_idx, n_verts: int, dim: int, out=None, prec="mixed", stream=None):
    """Assembly E^T of element vectors [(dim+1)*n_comp][C] into nodal values [n_comp][V]."""
    p = precision(prec)
    dt = value_dtype(p)
    rows, C = int(elem.shape[0]), int(elem.shape[1])
    n_comp = rows // (dim + 1)
    if n_comp * (dim + 1) != rows:
        raise ValueError("elem rows must be a multiple of dim+1")
    dev = elem.device
    out = torch.empty((n_comp, n_verts), dtype=dt, device=dev) if out is None else out
    st = lib().fem_gather_nodes(dim, n_comp, C, n_verts, _dev(elem, "elem", dt, None, dev),
                                _dev(node_ptr, "node_ptr", torch.int32, (n_verts + 1,), dev),
                                _dev(node_idx, "node_idx", torch.int32, ((dim + 1) * C,), dev),
                                _dev(out, "out", dt, (n_comp, n_verts), dev), p, _stream(stream))
    _check("fem_gather_nodes", st)
    return out


def fem_check_mesh(coords, conn, counts=None, stream=None) -> torch.Tensor:
    """Device int64[4]: bad vertex ids, degenerate cells, mixed-form fallback cells, inverted cells."""
    dim, V, C = _mesh_sizes(coords, conn)
    dev = coords.device
    counts = torch.empty(4, dtype=torch.int64, device=dev) if counts is None else counts
    st = lib().fem_check_mesh(dim, C, V, _dev(coords, "coords", torch.float64, device=dev),
                              _dev(conn, "conn", torch.int32, device=dev),
                              _dev(counts, "counts", torch.int64, (4,), dev), _stream(stream))
    _check("fem_check_mesh", st)
    return counts


def fem_probe(kind: int, n_threads: int, iters: int, out=None, stream=None) -> torch.Tensor:
    dt = torch.float64 if kind == 0 else torch.float32
    out = torch.empty(n_threads, dtype=dt, device="cuda") if out is None else out
    st = lib().fem_probe(kind, n_threads, iters, _dev(out, "out", dt, (n_threads,)), _stream(stream))
    _check("fem_probe", st)
    return out


def fem_device_error(stream=None) -> int:
    """Synchronise `stream`; return (and clear) the device error status: 0 (FEM_OK), -6
    (FEM_ERR_TIMEOUT) when a kernel gave up a bounded device-side wait, or -5
    (FEM_ERR_BADMESH) when a kernel met a vertex id outside [0, n_verts) or a degenerate
    cell (det J = 0, non-finite, or a repeated vertex id)."""
    return int(lib().fem_device_error(_stream(stream)))


def fem_selftest_quotient(num: torch.Tensor, den: torch.Tensor, stream=None):
    """(library quotient num / |den|, IEEE num / fabs(den)) computed on the device."""
    n = int(num.numel())
    if den.numel() != n:
        raise ValueError("num and den differ in size")
    q_lib = torch.empty_like(num)
    q_ieee = torch.empty_like(num)
    _check("fem_selftest_quotient", lib().fem_selftest_quotient(
        n, _dev(num, "num", torch.float64), _dev(den, "den", torch.float64), _dev(q_lib, "q_lib", torch.float64),
        _dev(q_ieee, "q_ieee", torch.float64), _stream(stream)))
    return q_lib, q_ieee


def fem_selftest_wait(budget_ns: int, stream=None) -> None:
    """Launch the bounded-wait self-test (a wait that can never succeed, `budget_ns` long)."""
    _check("fem_selftest_wait", lib().fem_selftest_wait(int(budget_ns), _stream(stream)))


def fem_set_mixed_threshold(tau: float) -> None:
    _check("fem_set_mixed_threshold", lib().fem_set_mixed_threshold(float(tau)))


def fem_get_mixed_threshold() -> float:
    return float(lib().fem_get_mixed_threshold())


def fem_version() -> str:
    return lib().fem_version().decode()


def fem_status_string(st: int) -> str:
    return lib().fem_status_string(int(st)).decode()
