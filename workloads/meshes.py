"""Jittered structured simplex meshes of the unit square and the unit cube.

Layout (shared by every consumer):
  coords : float64, shape (dim, V)   -- structure of arrays, vertex index fastest
  conn   : int32,   shape (dim+1, C) -- structure of arrays, cell index fastest

Vertices are numbered lexicographically (x fastest) and cells follow the order of
the grid squares/hexes they split, so consecutive cells share vertices; this keeps
the vertex gathers of consecutive cells close in memory.

Every cell is generated with a positive orientation (det J > 0 before jitter);
the jitter amplitudes used by the workloads keep it positive, which the tests check.
"""

from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Mesh:
    dim: int
    coords: np.ndarray  # (dim, V) float64
    conn: np.ndarray  # (dim+1, C) int32

    @property
    def n_verts(self) -> int:
        return int(self.coords.shape[1])

    @property
    def n_cells(self) -> int:
        return int(self.conn.shape[1])


def _rng(seed: int) -> np.random.Generator:
    # Philox is a counter-based generator with a published definition.
    return np.random.Generator(np.random.Philox(seed))


def square_mesh(nx: int, ny: int | None = None, jitter: float = 0.2, seed: int = 0) -> Mesh:
    """Unit square split into nx*ny rectangles, each cut into two triangles along
    the (0,0)-(1,1) diagonal: 2*nx*ny cells, (nx+1)*(ny+1) vertices.

    Interior vertices move by U[-jitter*hx, jitter*hx] in x and U[-jitter*hy, jitter*hy]
    in y (seeded). Boundary vertices stay on the boundary.
    """
    ny = nx if ny is None else ny
    hx, hy = 1.0 / nx, 1.0 / ny
    i = np.arange(nx + 1, dtype=np.float64)
    j = np.arange(ny + 1, dtype=np.float64)
    X, Y = np.meshgrid(i * hx, j * hy, indexing="xy")  # (ny+1, nx+1): x fastest
    x = X.ravel().copy()
    y = Y.ravel().copy()
    if jitter:
        rng = _rng(seed)
        jx = rng.uniform(-jitter * hx, jitter * hx, size=x.shape)
        jy = rng.uniform(-jitter * hy, jitter * hy, size=y.shape)
        ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
        interior = ((ii > 0) & (ii < nx) & (jj > 0) & (jj < ny)).ravel()
        x[interior] += jx[interior]
        y[interior] += jy[interior]
    coords = np.stack([x, y])

    si, sj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    si = si.ravel().astype(np.int64)
    sj = sj.ravel().astype(np.int64)
    v00 = si + (nx + 1) * sj
    v10 = v00 + 1
    v01 = v00 + (nx + 1)
    v11 = v01 + 1
    C = 2 * nx * ny
    conn = np.empty((3, C), dtype=np.int32)
    # lower-right triangle (v00, v10, v11) and upper-left triangle (v00, v11, v01),
    # both counter-clockwise
    conn[0, 0::2], conn[1, 0::2], conn[2, 0::2] = v00, v10, v11
    conn[0, 1::2], conn[1, 1::2], conn[2, 1::2] = v00, v11, v01
    return Mesh(2, coords, conn)


# Kuhn (Freudenthal) split of a hex into 6 tets sharing the diagonal v000-v111: for
# every permutation p of the axes, the path v000 -> +e_p0 -> +e_p1 -> +e_p2 = v111.
# The determinant of that path equals sign(p); odd permutations swap the middle two
# vertices so that every tet is positively oriented.
_PERMS = [(0, 1, 2, +1), (0, 2, 1, -1), (1, 0, 2, -1), (1, 2, 0, +1), (2, 0, 1, +1), (2, 1, 0, -1)]


def cube_mesh(n: int, jitter: float = 0.15, seed: int = 0) -> Mesh:
    """Unit cube as n^3 hexes, each split into 6 tets: 6*n^3 cells, (n+1)^3 vertices.

    Interior vertices move by U[-jitter*h, jitter*h] per coordinate (seeded).
    """
    h = 1.0 / n
    m = n + 1
    g = np.arange(m, dtype=np.float64) * h
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")  # X fastest in ravel order
    coords = np.stack([X.ravel(), Y.ravel(), Z.ravel()]).copy()
    if jitter:
        rng = _rng(seed)
        jit = rng.uniform(-jitter * h, jitter * h, size=coords.shape)
        kk, jj, ii = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
        interior = (
            (ii > 0) & (ii < n) & (jj > 0) & (jj < n) & (kk > 0) & (kk < n)
        ).ravel()
        coords[:, interior] += jit[:, interior]

    hk, hj, hi = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    base = (hi + m * hj + m * m * hk).ravel().astype(np.int64)
    stride = np.array([1, m, m * m], dtype=np.int64)
    C = 6 * n ** 3
    conn = np.empty((4, C), dtype=np.int32)
    for t, (p0, p1, p2, sgn) in enumerate(_PERMS):
        a = base
        b = base + stride[p0]
        c = b + stride[p1]
        d = base + stride.sum()
        if sgn < 0:
            b, c = c, b
        conn[0, t::6], conn[1, t::6], conn[2, t::6], conn[3, t::6] = a, b, c, d
    return Mesh(3, coords, conn)


def first_cells(mesh: Mesh, n_cells: int) -> Mesh:
    """The first n_cells cells (in generation order), with the vertex arrays trimmed
    to the highest vertex index those cells use."""
    if n_cells > mesh.n_cells:
        raise ValueError(f"mesh has {mesh.n_cells} cells, asked for {n_cells}")
    conn = np.ascontiguousarray(mesh.conn[:, :n_cells])
    nv = int(conn.max()) + 1 if n_cells else 0
    coords = np.ascontiguousarray(mesh.coords[:, :nv])
    return Mesh(mesh.dim, coords, conn)


def smallest_cube_for(n_cells: int) -> int:
    """Smallest n with 6*n^3 >= n_cells."""
    n = max(1, int(round((n_cells / 6.0) ** (1.0 / 3.0))) - 1)
    while 6 * n ** 3 < n_cells:
        n += 1
    return n


def smallest_square_for(n_cells: int) -> int:
    """Smallest n with 2*n^2 >= n_cells."""
    n = max(1, int(round((n_cells / 2.0) ** 0.5)) - 1)
    while 2 * n * n < n_cells:
        n += 1
    return n
