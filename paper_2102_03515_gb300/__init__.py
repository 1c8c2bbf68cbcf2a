"""GB300 solver for the P1 finite element system (rho K + M) u = f of arXiv 2102.03515.

This package is a thin ctypes binding of the CUDA library ``_lib/libfemamg.so`` (C ABI in
``include/femamg.h``).  Every step of the solver runs in the library's kernels; this
module only marshals arguments (torch tensors as device buffers, torch streams).  If the
library is missing the import of any entry point raises: there is no fallback.

A solve at h = 1/n with rho = h^2 and the smooth target of Sec. 4.1::

    import torch, paper_2102_03515_gb300 as fa
    n = 128
    sys_ = fa.fem_assemble(n, 1.0 / n ** 2, {"kind": "sine"})
    h = fa.amg_setup(sys_, precision=fa.AMG_PREC_FP32)      # FP32 V-cycle
    u = torch.zeros((n - 1) ** 3, dtype=torch.float64, device="cuda")
    res = fa.pcg_solve(sys_, h, None, u, tol=1e-8)[0]         # flexible CG, FP64
    err = fa.fem_errors(sys_, u, {"kind": "sine"})            # ||ubar - u_h||^2 in L2, H1
    hm1 = fa.fem_error_hm1(sys_, u, {"kind": "sine"})         # ... in the discrete H^-1
    fa.amg_hier_destroy(h)
    fa.fem_system_destroy(sys_)
"""
from __future__ import annotations

from ._binding import (  # noqa: F401
    AMG_COARSEN_RED_BLACK, AMG_COARSEN_SA, AMG_ORDER_HASH, AMG_ORDER_NATURAL, AMG_PREC_BF16,
    AMG_PREC_FP32, AMG_PREC_FP64,
    AMG_SMOOTHER_CHEBYSHEV, AMG_SMOOTHER_L1_JACOBI, AMG_SMOOTHER_SGS, FEM_FMT_AUTO, FEM_FMT_CSR,
    FEM_FMT_STENCIL, FemError, PCG_STOP_PRECONDITIONED, PCG_STOP_RESIDUAL, amg_default_opts,
    amg_hier_destroy, amg_hier_export, amg_hier_get_info, amg_setup, amg_vcycle,
    amg_galerkin_timed, amg_vcycle_graph, bddc_destroy, bddc_get_setup_ms, bddc_setup,
    bddc_solve, fem_assemble, fem_bddc_partition, make_allreduce,
    fem_assemble_mesh, fem_assemble_on_mesh, fem_error_indicator, fem_mark_bulk,
    fem_mesh_create, fem_mesh_destroy, fem_mesh_download, fem_mesh_get_info, fem_mesh_refine,
    fem_assemble_rhs, fem_assemble_rhs_noalloc, fem_autotune_clear, fem_autotune_pin,
    fem_autotune_report, fem_error_hm1, fem_errors, fem_kernel_launches, fem_last_error,
    fem_measure_fp64_rate, fem_recover, fem_spmv, fem_spmv_timed,
    fem_system_destroy, fem_system_dof_vertices, fem_system_export, fem_system_get_info,
    fem_system_get_rhs, fem_version,
    lib, pcg_batch_admit, pcg_batch_create, pcg_batch_destroy, pcg_batch_footprint,
    pcg_batch_poll, pcg_batch_retire, pcg_batch_step, pcg_default_opts, pcg_solve,
)
