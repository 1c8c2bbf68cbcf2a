"""GB300 solver for the P1 finite element system (rho K + M) u = f of arXiv 2102.03515.

This package is a thin ctypes binding of the CUDA library ``_lib/libfemamg.so`` (C ABI in
``include/femamg.h``).  Every step of the solver runs in the library's kernels; this
module only marshals arguments (torch tensors as device buffers, torch streams).  If the
library is missing the import of any entry point raises: there is no fallback.
"""
from __future__ import annotations

from ._binding import (  # noqa: F401
    AMG_COARSEN_RED_BLACK, AMG_COARSEN_SA, AMG_PREC_BF16, AMG_PREC_FP32, AMG_PREC_FP64,
    AMG_SMOOTHER_CHEBYSHEV, AMG_SMOOTHER_L1_JACOBI, AMG_SMOOTHER_SGS, FEM_FMT_AUTO, FEM_FMT_CSR,
    FEM_FMT_STENCIL, FemError, PCG_STOP_PRECONDITIONED, PCG_STOP_RESIDUAL, amg_default_opts,
    amg_hier_destroy, amg_hier_export, amg_hier_get_info, amg_setup, amg_vcycle,
    amg_vcycle_graph, fem_assemble,
    fem_assemble_mesh, fem_assemble_on_mesh, fem_error_indicator, fem_mark_bulk,
    fem_mesh_create, fem_mesh_destroy, fem_mesh_download, fem_mesh_get_info, fem_mesh_refine,
    fem_assemble_rhs, fem_assemble_rhs_noalloc, fem_autotune_clear, fem_autotune_pin,
    fem_autotune_report, fem_error_hm1, fem_errors, fem_kernel_launches, fem_last_error,
    fem_measure_fp64_rate, fem_recover, fem_spmv,
    fem_system_destroy, fem_system_dof_vertices, fem_system_export, fem_system_get_info,
    fem_system_get_rhs, fem_version,
    lib, pcg_batch_admit, pcg_batch_create, pcg_batch_destroy, pcg_batch_footprint,
    pcg_batch_poll, pcg_batch_retire, pcg_batch_step, pcg_default_opts, pcg_solve,
)
