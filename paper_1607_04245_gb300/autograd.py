"""torch.autograd.Function for the Laplacian element residual.

forward  : r = fem_integrate_laplacian(u, K)            (element vectors [dim+1][C])
backward : for an incoming gradient lambda = dL/dr, the hand-written adjoint kernels
           of fem_adjoint_laplacian return dL/dK (per quadrature point) and dL/du
           (per vertex, summed over the vertex-to-cell lists in a fixed order).

Like every call of the library, the kernels report a bounded device-side wait that gave up,
or a bad mesh, through the device error word rather than an exception: a training loop that
needs the guarantee calls fem_device_error() (one synchronisation) after its steps.
"""

from __future__ import annotations

import numpy as np
import torch

from .binding import fem_adjoint_laplacian, fem_build_node2cell, fem_integrate_laplacian


class DeviceMesh:
    """A mesh resident on the device with its quadrature rule and vertex-to-cell lists."""

    def __init__(self, coords: torch.Tensor, conn: torch.Tensor, qpts, qw, build_lists: bool = True):
        self.coords = coords.contiguous()
        self.conn = conn.contiguous()
        self.dim = int(coords.shape[0])
        self.n_verts = int(coords.shape[1])
        self.n_cells = int(conn.shape[1])
        self.qpts = np.ascontiguousarray(qpts, dtype=np.float64)
        self.qw = np.ascontiguousarray(qw, dtype=np.float64)
        self.node_ptr = self.node_idx = None
        if build_lists:
            self.node_ptr, self.node_idx = fem_build_node2cell(self.conn, self.n_verts)

    @property
    def n_q(self) -> int:
        return int(self.qw.shape[0])


class LaplacianResidual(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, K, mesh: DeviceMesh, prec: str):
        r = fem_integrate_laplacian(mesh.coords, mesh.conn, u.contiguous(), K.contiguous(), mesh.qpts, mesh.qw,
                                    prec=prec)
        ctx.save_for_backward(u, K)
        ctx.mesh = mesh
        ctx.prec = prec
        return r

    @staticmethod
    def backward(ctx, grad_r):
        u, K = ctx.saved_tensors
        mesh = ctx.mesh
        if mesh.node_ptr is None:
            mesh.node_ptr, mesh.node_idx = fem_build_node2cell(mesh.conn, mesh.n_verts)
        dK, du = fem_adjoint_laplacian(mesh.coords, mesh.conn, u.contiguous(), K.contiguous(), mesh.qpts, mesh.qw,
                                       grad_r.contiguous(), mesh.node_ptr, mesh.node_idx, prec=ctx.prec)
        return (du if ctx.needs_input_grad[0] else None, dK if ctx.needs_input_grad[1] else None, None, None)


def laplacian_residual(u: torch.Tensor, K: torch.Tensor, mesh: DeviceMesh, prec: str = "fp64") -> torch.Tensor:
    """Element residuals of the variable-coefficient Laplacian, differentiable in u and K."""
    return LaplacianResidual.apply(u, K, mesh, prec)
