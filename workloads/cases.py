"""Complete seeded problem instances: mesh + quadrature + nodal field + coefficients.

Recipes (sizes are parameters; the defaults are the full workloads):

  laplacian_square_case  2D P1 Laplacian: 64x64 squares -> 8192 triangles, interior
                         jitter +-0.2h, 3-point rule, K(x) = 1 + 0.5 sin(2 pi x) cos(2 pi y)
                         at the physical quadrature points, nodal u ~ U[-1, 1].
  laplacian_cube_case    3D P1 Laplacian: 64^3 hexes x 6 -> 1,572,864 tets, jitter +-0.15h,
                         4-point rule, K ~ lognormal(0, 1) i.i.d. per quadrature point,
                         nodal u ~ U[-1, 1].  A smaller cell count takes the first C cells
                         of the smallest n^3 x 6 mesh holding at least C cells.
  elasticity_case        P1 linear elasticity: 2D 2048x1024 squares -> 2^22 triangles;
                         3D the first 2^21 tets of a 71^3 x 6 mesh.  Per quadrature point
                         E ~ lognormal(0, 0.5), nu ~ U[0.2, 0.45], converted to the Lame
                         pair (lambda, mu) with the plane-strain/3D formulas; nodal
                         displacements N(0, sigma = 1e-2) per component.
  adjoint_case           the 3D Laplacian case plus an adjoint weight per element dof,
                         U[-1, 1], shape (d+1, C).
  reaction_inputs        for a case: an auxiliary P1 field a ~ lognormal(0, 0.5) per vertex
                         and a reaction coefficient c ~ U[0.5, 2] per quadrature point.
  dirichlet_problem      for a case: boundary vertices of the unit square/cube held at the
                         linear function g(x) = 1 + 2 x_1 - 3 x_2 (+ 0.5 x_3), zero initial
                         guess inside.

Random streams: numpy's Philox generator, one independent stream per array, all
derived from one integer seed, so every consumer sees identical arrays.
"""

from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

from .meshes import Mesh, cube_mesh, first_cells, smallest_cube_for, smallest_square_for, square_mesh
from .quadrature import QuadRule, rule_for_dim


@dataclasses.dataclass
class Case:
    physics: str  # "laplacian" or "elasticity"
    mesh: Mesh
    rule: QuadRule
    u: np.ndarray  # laplacian: (V,), elasticity: (dim, V); float64
    K: Optional[np.ndarray] = None  # (n_q, C) float64
    lam: Optional[np.ndarray] = None  # (n_q, C) float64
    mu: Optional[np.ndarray] = None  # (n_q, C) float64
    adj: Optional[np.ndarray] = None  # (dim+1, C) adjoint weights, float64
    name: str = ""

    @property
    def dim(self) -> int:
        return self.mesh.dim

    @property
    def n_cells(self) -> int:
        return self.mesh.n_cells

    @property
    def n_verts(self) -> int:
        return self.mesh.n_verts

    @property
    def n_comp(self) -> int:
        return 1 if self.physics == "laplacian" else self.dim

    def rounded_to_f32(self) -> "Case":
        """The same case with every value array rounded to float32 and widened back
        to float64. Coordinates and quadrature tables stay float64 (they are always
        passed in double precision)."""
        r = lambda a: None if a is None else a.astype(np.float32).astype(np.float64)
        return dataclasses.replace(
            self, u=r(self.u), K=r(self.K), lam=r(self.lam), mu=r(self.mu), adj=r(self.adj)
        )


def _streams(seed: int, n: int):
    return [np.random.Generator(np.random.Philox(s)) for s in np.random.SeedSequence(seed).spawn(n)]


def physical_quad_points(mesh: Mesh, rule: QuadRule) -> np.ndarray:
    """Physical position of every quadrature point, shape (n_q, dim, C): the image of
    the reference point under the cell's affine map, written as the barycentric
    combination sum_b beta_b(xi_q) x_b with beta = (1 - sum xi, xi_1, ..., xi_d).
    Used only to sample a coefficient field defined as a function of x."""
    d = mesh.dim
    bary = np.concatenate([1.0 - rule.points.sum(axis=1, keepdims=True), rule.points], axis=1)  # (n_q, d+1)
    verts = mesh.coords[:, mesh.conn]  # (d, d+1, C)
    return np.einsum("qb,ibc->qic", bary, verts)


def laplacian_square_case(n: int = 64, jitter: float = 0.2, seed: int = 0) -> Case:
    s_u, = _streams(seed, 1)
    mesh = square_mesh(n, n, jitter=jitter, seed=seed)
    rule = rule_for_dim(2)
    xq = physical_quad_points(mesh, rule)
    K = 1.0 + 0.5 * np.sin(2 * np.pi * xq[:, 0, :]) * np.cos(2 * np.pi * xq[:, 1, :])
    u = s_u.uniform(-1.0, 1.0, size=mesh.n_verts)
    return Case("laplacian", mesh, rule, u, K=np.ascontiguousarray(K), name=f"lap2d_{2*n*n}")


def _cube_cells(n_cells: int, jitter: float, seed: int, n: Optional[int] = None) -> Mesh:
    n = smallest_cube_for(n_cells) if n is None else n
    mesh = cube_mesh(n, jitter=jitter, seed=seed)
    return mesh if mesh.n_cells == n_cells else first_cells(mesh, n_cells)


def laplacian_cube_case(n_cells: int = 1572864, jitter: float = 0.15, seed: int = 0) -> Case:
    s_u, s_k = _streams(seed, 2)
    mesh = _cube_cells(n_cells, jitter, seed)
    rule = rule_for_dim(3)
    K = s_k.lognormal(0.0, 1.0, size=(rule.n_q, mesh.n_cells))
    u = s_u.uniform(-1.0, 1.0, size=mesh.n_verts)
    return Case("laplacian", mesh, rule, u, K=K, name=f"lap3d_{n_cells}")


def lame_from_young_poisson(E: np.ndarray, nu: np.ndarray):
    """Lame parameters from Young's modulus and Poisson's ratio (3D / plane strain)."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def elasticity_case(dim: int, n_cells: Optional[int] = None, jitter: Optional[float] = None,
                    seed: int = 0) -> Case:
    s_u, s_e, s_nu = _streams(seed, 3)
    rule = rule_for_dim(dim)
    if dim == 2:
        n_cells = 1 << 22 if n_cells is None else n_cells
        jitter = 0.2 if jitter is None else jitter
        if n_cells == 1 << 22:
            mesh = square_mesh(2048, 1024, jitter=jitter, seed=seed)
        else:
            m = smallest_square_for(n_cells)
            mesh = square_mesh(m, m, jitter=jitter, seed=seed)
            if mesh.n_cells != n_cells:
                mesh = first_cells(mesh, n_cells)
    elif dim == 3:
        n_cells = 1 << 21 if n_cells is None else n_cells
        jitter = 0.15 if jitter is None else jitter
        mesh = _cube_cells(n_cells, jitter, seed, n=71 if n_cells == 1 << 21 else None)
    else:
        raise ValueError("dim must be 2 or 3")
    E = s_e.lognormal(0.0, 0.5, size=(rule.n_q, mesh.n_cells))
    nu = s_nu.uniform(0.2, 0.45, size=(rule.n_q, mesh.n_cells))
    lam, mu = lame_from_young_poisson(E, nu)
    u = s_u.normal(0.0, 1e-2, size=(dim, mesh.n_verts))
    return Case("elasticity", mesh, rule, u, lam=lam, mu=mu, name=f"elast{dim}d_{n_cells}")


def adjoint_case(n_cells: int = 1572864, jitter: float = 0.15, seed: int = 0) -> Case:
    case = laplacian_cube_case(n_cells, jitter, seed)
    s_adj, = _streams(seed + 7919, 1)
    case.adj = s_adj.uniform(-1.0, 1.0, size=(case.dim + 1, case.n_cells))
    case.name = f"adj3d_{n_cells}"
    return case


def adjoint_weights(case: Case, seed: int = 7919) -> np.ndarray:
    s_adj, = _streams(seed, 1)
    return s_adj.uniform(-1.0, 1.0, size=(case.n_comp * (case.dim + 1), case.n_cells))


SERVING_PHYSICS = (("laplacian", 2), ("laplacian", 3), ("elasticity", 2), ("elasticity", 3))


def serving_specs(n: int = 500, seed: int = 0, min_cells: int = 1000, max_cells: int = 1_000_000):
    """Request mix of the serving stream: physics uniform over {2D, 3D} x {Laplacian,
    elasticity}; Laplacian requests are a residual or an adjoint evaluation with equal
    probability (elasticity: residual); cell counts log-uniform in [min_cells, max_cells];
    a fresh seed per request."""
    rng = np.random.Generator(np.random.Philox(np.random.SeedSequence(seed).spawn(1)[0]))
    specs = []
    for i in range(n):
        physics, dim = SERVING_PHYSICS[int(rng.integers(0, 4))]
        kind = "adjoint" if physics == "laplacian" and rng.random() < 0.5 else "residual"
        C = int(round(np.exp(rng.uniform(np.log(min_cells), np.log(max_cells)))))
        specs.append({"rid": i, "physics": physics, "dim": dim, "kind": kind, "n_cells": C,
                      "seed": int(seed) * 1_000_003 + i + 1})
    return specs


def serving_case(spec) -> Case:
    """The case of one serving request: the first C cells of the smallest grid mesh that
    holds them (jitter, coefficients and fields as in the other workloads)."""
    C, dim, s = spec["n_cells"], spec["dim"], spec["seed"]
    if spec["physics"] == "elasticity":
        case = elasticity_case(dim, C, seed=s)
    elif dim == 2:
        m = smallest_square_for(C)
        base = laplacian_square_case(m, seed=s)
        mesh = first_cells(base.mesh, C) if base.n_cells != C else base.mesh
        case = Case("laplacian", mesh, base.rule, base.u[: mesh.n_verts], K=np.ascontiguousarray(base.K[:, :C]))
    else:
        case = laplacian_cube_case(C, seed=s)
    if spec["kind"] == "adjoint":
        s_adj, = _streams(s + 7919, 1)
        case.adj = s_adj.uniform(-1.0, 1.0, size=(case.dim + 1, case.n_cells))
    case.name = f"req{spec['rid']}_{spec['physics']}{dim}d_{spec['kind']}_{C}"
    return case


def reaction_inputs(case: Case, seed: int = 0):
    """(a, c): a P1 auxiliary field a[V] ~ lognormal(0, 0.5) and a reaction coefficient
    c[n_q][C] ~ U[0.5, 2] for the case's mesh and rule."""
    s_a, s_c = _streams(seed + 104729, 2)
    a = s_a.lognormal(0.0, 0.5, size=case.n_verts)
    c = s_c.uniform(0.5, 2.0, size=(case.rule.n_q, case.n_cells))
    return a, c


def dirichlet_problem(case: Case):
    """(fixed, x0): the vertices on the boundary of the unit square/cube (uint8 mask) and
    an initial vector holding g(x) = 1 + 2 x_1 - 3 x_2 (+ 0.5 x_3) there and 0 inside."""
    x = case.mesh.coords
    fixed = np.any((np.abs(x) < 1e-14) | (np.abs(x - 1.0) < 1e-14), axis=0)
    coef = np.array([2.0, -3.0, 0.5])[: case.dim]
    g = 1.0 + coef @ x
    return fixed.astype(np.uint8), np.where(fixed, g, 0.0)
