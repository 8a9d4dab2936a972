"""GB300 ghost-cell immersed-boundary pressure Poisson library (Python binding).

The compute path is the CUDA library ``lib/libibmpoisson.so`` (built by
``paper_2605_04335_gb300.build``); this package only marshals arguments to its C ABI
(``include/ibm_poisson.h``).  Import of the binding fails loudly if the library is
missing: there is no CPU fallback.
"""
from .ibm import (IbmError, Context, Tables, SolveOpts, ibm_ctx_create, ibm_ctx_destroy, ibm_classify,
                  ibm_tables_counts, ibm_tables_export, ibm_tables_destroy, poisson_solve, load_library,
                  library_path, ibm_smoother_sweeps, ibm_smoother_sweeps_timed, ibm_ctx_launch_count,
                  ibm_ctx_set_sweep_wait_limit, ibm_smoother_apply, ibm_measure_fp64_rate,
                  ibm_residual_norm_noalloc, poisson_solve_batched,
                  ibm_autotune, ibm_reclassify,
                  ibm_set_neumann, ibm_neumann_rigid, ibm_surface_forces, HelmholtzOpts,
                  ibm_helmholtz_solve, ibm_boundary_velocity_rigid, ibm_helmholtz_sweeps_timed)

__all__ = ["IbmError", "Context", "Tables", "SolveOpts", "ibm_ctx_create", "ibm_ctx_destroy", "ibm_classify",
           "ibm_tables_counts", "ibm_tables_export", "ibm_tables_destroy", "poisson_solve", "load_library",
           "library_path", "ibm_smoother_sweeps", "ibm_smoother_sweeps_timed", "ibm_ctx_launch_count",
           "ibm_ctx_set_sweep_wait_limit", "ibm_smoother_apply", "ibm_measure_fp64_rate",
           "ibm_residual_norm_noalloc", "poisson_solve_batched", "ibm_autotune", "ibm_reclassify",
           "ibm_set_neumann", "ibm_neumann_rigid", "ibm_surface_forces", "HelmholtzOpts",
           "ibm_helmholtz_solve", "ibm_boundary_velocity_rigid", "ibm_helmholtz_sweeps_timed"]
