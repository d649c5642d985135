"""Helpers shared by the GPU parity tests: move a seeded case to the device in a given
precision form and compare against the oracle."""

from __future__ import annotations

import numpy as np
import torch

import paper_1607_04245_gb300 as fem

# relative max-norm tolerances: ||r_gpu - r_oracle||_inf / ||r_oracle||_inf
#   fp64   1e-12: the float64 form
#   mixed  2e-5 : float32 storage with compensated coordinate differences, float64 fallback
#   fp32   1e-3 : the plain float32 ablation; its error grows like 2^-24 |x| / h (coordinates
#                 rounded before the Jacobian), about 1e-4 on a 2048 x 1024 grid
TOL = {"fp64": 1e-12, "mixed": 2e-5, "fp32": 1e-3}
PRECS = ("fp64", "mixed", "fp32")


def as_input(case, prec):
    """The case whose value arrays hold exactly what the device sees (float32-rounded for
    the float32 forms), so the oracle and the kernel integrate identical data."""
    return case if prec == "fp64" else case.rounded_to_f32()


def to_dev(a, dtype, device="cuda"):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=dtype)


def device_arrays(case, prec, device="cuda"):
    c = as_input(case, prec)
    dt = fem.value_dtype(prec)
    d = {
        "coords": to_dev(c.mesh.coords, torch.float64, device),
        "conn": to_dev(c.mesh.conn, torch.int32, device),
        "u": to_dev(c.u, dt, device),
    }
    for name in ("K", "lam", "mu", "adj"):
        a = getattr(c, name)
        if a is not None:
            d[name] = to_dev(a, dt, device)
    return c, d


def rel_err(gpu, ref) -> float:
    g = gpu.double().cpu().numpy() if isinstance(gpu, torch.Tensor) else np.asarray(gpu, dtype=np.float64)
    scale = np.abs(ref).max()
    return float(np.abs(g - ref).max() / scale) if scale > 0 else float(np.abs(g).max())


def residual(case, d, prec, out=None, stream=None):
    q = case.rule
    if case.physics == "laplacian":
        return fem.fem_integrate_laplacian(d["coords"], d["conn"], d["u"], d["K"], q.points, q.weights,
                                           out=out, prec=prec, stream=stream)
    return fem.fem_integrate_elasticity(d["coords"], d["conn"], d["u"], d["lam"], d["mu"], q.points, q.weights,
                                        out=out, prec=prec, stream=stream)


def misaligned(t: torch.Tensor) -> torch.Tensor:
    """A contiguous copy of t whose storage starts one element past a 16-byte boundary."""
    flat = torch.empty(t.numel() + 1, dtype=t.dtype, device=t.device)
    v = flat[1:].view(t.shape)
    v.copy_(t)
    assert v.data_ptr() % 16 != 0
    return v
