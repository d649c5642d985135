"""GB300-native batched quadrature-based P1 element integration.

Knepley, Rupp, Terrel, "Finite Element Integration with Quadrature on the GPU":
per-cell element residuals of the variable-coefficient Laplacian and of linear
elasticity (Eq. 2 with f0 = 0), their adjoint, and a continuous-batching server,
all computed by the CUDA C-ABI library libfem (include/fem.h). The Python layer
only marshals arguments; importing it does not load the library, the first call
does, and fails loudly if the library has not been built.
"""

from .binding import (  # noqa: F401
    FEM_FP32,
    FEM_FP32_MIXED,
    FEM_FP64,
    FEM_FP64_DF,
    FEM_MAX_QPTS,
    FemError,
    PreparedCall,
    fem_adjoint_laplacian,
    fem_build_node2cell,
    fem_check_mesh,
    fem_device_error,
    fem_element_values,
    fem_gather_nodes,
    fem_get_mixed_threshold,
    fem_integrate_elasticity,
    fem_host_work_bytes,
    fem_integrate_laplacian,
    fem_integrate_laplacian_fields,
    fem_integrate_laplacian_host,
    fem_integrate_laplacian_geom,
    fem_integrate_laplacian_transposed,
    fem_integrate_pointwise,
    fem_integrate_laplacian_prepared,
    prepared_integrate_elasticity,
    prepared_integrate_laplacian,
    fem_prepare_vertices,
    fem_integrate_reaction_diffusion,
    fem_precompute_geometry,
    fem_pcg_elasticity,
    fem_pcg_elasticity_refined,
    fem_pcg_laplacian,
    fem_pcg_laplacian_refined,
    fem_probe,
    fem_selftest_quotient,
    fem_selftest_wait,
    fem_set_mixed_threshold,
    fem_status_string,
    fem_version,
    precision,
    value_dtype,
)

__version__ = "0.1.0"
