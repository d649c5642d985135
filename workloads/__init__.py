"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This package generates meshes, quadrature tables, coefficient fields and request
streams. It holds none of the integration method's arithmetic: no Jacobians, no
gradients, no contractions. Both the CPU oracle and the CUDA library receive the
arrays it produces as plain inputs.

The paper measures on unstructured Triangle/TetGen meshes of the unit square and
cube (Sec. 6); those meshes are not available, so jittered structured simplex
meshes of the same domains stand in for them.
"""

from .meshes import Mesh, square_mesh, cube_mesh, first_cells, smallest_cube_for
from .quadrature import QuadRule, triangle_deg2, tetrahedron_deg2, rule_for_dim
from .cases import (
    Case,
    laplacian_square_case,
    laplacian_cube_case,
    elasticity_case,
    adjoint_case,
    lame_from_young_poisson,
    reaction_inputs,
    dirichlet_problem,
)

__all__ = [
    "reaction_inputs",
    "dirichlet_problem",
    "Mesh",
    "square_mesh",
    "cube_mesh",
    "first_cells",
    "smallest_cube_for",
    "QuadRule",
    "triangle_deg2",
    "tetrahedron_deg2",
    "rule_for_dim",
    "Case",
    "laplacian_square_case",
    "laplacian_cube_case",
    "elasticity_case",
    "adjoint_case",
    "lame_from_young_poisson",
]
