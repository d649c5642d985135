"""Host-buffer entry point: integrate arrays that live in host memory.

HostIntegrator keeps pinned host staging buffers and a device workspace. The Laplacian
goes through libfem's host entry (fem_integrate_laplacian_host): the vertex arrays are
uploaded once per call; by default (chunks = 0) the kernel then reads the connectivity and
coefficient rows from the pinned host buffers and writes the element vectors into a pinned
host buffer across the host link, so both directions stream for the whole kernel; with
chunks >= 1 the cells instead go through copy-engine transfers in chunks on two library
streams, overlapped with the kernels. Elasticity copies everything, runs the kernel and
copies back on one stream. This is the call a user with host data makes; the
benchmark's end-to-end figure is measured through it.
"""

from __future__ import annotations

from typing import Dict, Tuple

import numpy as np
import torch

from .binding import (fem_host_work_bytes, fem_integrate_elasticity, fem_integrate_laplacian_host, value_dtype)


class HostIntegrator:
    def __init__(self, device="cuda", stream: torch.cuda.Stream = None):
        self.device = torch.device(device)
        self.stream = stream or torch.cuda.Stream(device=self.device)
        self._dev: Dict[Tuple[str, tuple, torch.dtype], torch.Tensor] = {}
        self._pin: Dict[Tuple[str, tuple, torch.dtype], torch.Tensor] = {}
        self.h2d_bytes = 0
        self.d2h_bytes = 0

    def _buf(self, pool, key, shape, dtype, pinned):
        k = (key, tuple(shape), dtype)
        t = pool.get(k)
        if t is None:
            t = torch.empty(shape, dtype=dtype, pin_memory=True) if pinned else torch.empty(
                shape, dtype=dtype, device=self.device)
            pool[k] = t
        return t

    def pinned(self, key: str, a: np.ndarray, dtype: torch.dtype) -> torch.Tensor:
        """Stage a numpy array in a pinned host buffer (reused across calls)."""
        h = self._buf(self._pin, key, a.shape, dtype, True)
        h.numpy()[...] = a
        return h

    def _upload(self, key, host: torch.Tensor) -> torch.Tensor:
        d = self._buf(self._dev, key, host.shape, host.dtype, False)
        d.copy_(host, non_blocking=True)
        self.h2d_bytes += host.numel() * host.element_size()
        return d

    def laplacian(self, coords_h, conn_h, u_h, K_h, qpts, qw, prec="mixed", out_h=None, chunks=0) -> torch.Tensor:
        """All arguments are pinned host tensors (see pinned()); returns the element
        vectors in a pinned host tensor, valid after self.stream is synchronised."""
        dt = value_dtype(prec)
        dim, V = int(coords_h.shape[0]), int(coords_h.shape[1])
        C, nq = int(conn_h.shape[1]), int(K_h.shape[0])
        need = fem_host_work_bytes(dim, C, V, nq, prec, chunks)
        work = self._buf(self._dev, "host_work", (max(need, 1),), torch.uint8, False)
        if out_h is None:
            out_h = self._buf(self._pin, "out_h", (dim + 1, C), dt, True)
        fem_integrate_laplacian_host(coords_h, conn_h, u_h, K_h, qpts, qw, out_h, work, chunks=chunks, prec=prec,
                                     stream=self.stream)
        for t in (coords_h, conn_h, u_h, K_h):
            self.h2d_bytes += t.numel() * t.element_size()
        self.d2h_bytes += out_h.numel() * out_h.element_size()
        return out_h

    def elasticity(self, coords_h, conn_h, u_h, lam_h, mu_h, qpts, qw, prec="mixed", out_h=None) -> torch.Tensor:
        with torch.cuda.stream(self.stream):
            coords = self._upload("coords", coords_h)
            conn = self._upload("conn", conn_h)
            u = self._upload("u", u_h)
            lam = self._upload("lam", lam_h)
            mu = self._upload("mu", mu_h)
            dt = value_dtype(prec)
            dim = coords.shape[0]
            out = self._buf(self._dev, "out", ((dim + 1) * dim, conn.shape[1]), dt, False)
            fem_integrate_elasticity(coords, conn, u, lam, mu, qpts, qw, out=out, prec=prec, stream=self.stream)
            if out_h is None:
                out_h = self._buf(self._pin, "out_h", out.shape, dt, True)
            out_h.copy_(out, non_blocking=True)
            self.d2h_bytes += out.numel() * out.element_size()
        return out_h
