"""Quadrature tables on the reference simplex (vertices 0, e_1, ..., e_d).

The paper does not print its rules; the workloads call for a 3-point degree-2
rule on triangles and a 4-point degree-2 rule on tetrahedra. These are data passed
to both the oracle and the CUDA library across their interfaces.

  triangle:    interior points (1/6,1/6), (2/3,1/6), (1/6,2/3), weights 1/6 each
               (weights sum to the reference area 1/2; the edge-midpoint rule is
               also 3-point degree 2, the interior one is used here)
  tetrahedron: (a,a,a), (b,a,a), (a,b,a), (a,a,b) with a = (5 - sqrt 5)/20,
               b = (5 + 3 sqrt 5)/20, weights 1/24 each (sum = 1/6)
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class QuadRule:
    dim: int
    points: np.ndarray  # (n_q, dim) reference coordinates, float64, C order
    weights: np.ndarray  # (n_q,) float64

    @property
    def n_q(self) -> int:
        return int(self.weights.shape[0])


def triangle_deg2() -> QuadRule:
    p = np.array([[1 / 6, 1 / 6], [2 / 3, 1 / 6], [1 / 6, 2 / 3]], dtype=np.float64)
    w = np.full(3, 1 / 6, dtype=np.float64)
    return QuadRule(2, p, w)


def tetrahedron_deg2() -> QuadRule:
    a = (5.0 - math.sqrt(5.0)) / 20.0
    b = (5.0 + 3.0 * math.sqrt(5.0)) / 20.0
    p = np.array([[a, a, a], [b, a, a], [a, b, a], [a, a, b]], dtype=np.float64)
    w = np.full(4, 1 / 24, dtype=np.float64)
    return QuadRule(3, p, w)


def rule_for_dim(dim: int) -> QuadRule:
    if dim == 2:
        return triangle_deg2()
    if dim == 3:
        return tetrahedron_deg2()
    raise ValueError(f"dim must be 2 or 3, got {dim}")
