"""Run single kernels of the solver at full size, for profiler captures.

    python -m paper_2102_03515_gb300.profile_kernels spmv64 256    # FP64 stencil q = A p
    python -m paper_2102_03515_gb300.profile_kernels vcycle32 256  # one FP32 V-cycle
    python -m paper_2102_03515_gb300.profile_kernels step 256      # one assemble+setup+solve
    python -m paper_2102_03515_gb300.profile_kernels batched 128   # 64-slot batched solve
    python -m paper_2102_03515_gb300.profile_kernels galerkin 128  # finest Galerkin product
    python -m paper_2102_03515_gb300.profile_kernels cgop 256      # CG's q = A p

Each mode runs its work three times; the last pass is inside the NVTX range "profiled",
so that `ncu --nvtx --nvtx-include "profiled/"` sees only the steady state (the first
passes also tune the launch shapes).
"""
from __future__ import annotations

import contextlib
import sys

import torch

from . import _binding as fa


@contextlib.contextmanager
def _range(last: bool):
    if last:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("profiled")
    try:
        yield
    finally:
        if last:
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()


def main(argv):
    mode = argv[1] if len(argv) > 1 else "spmv64"
    n = int(argv[2]) if len(argv) > 2 else 256
    rho = 1.0 / n ** 2
    N = (n - 1) ** 3
    sine = {"kind": "sine"}
    reps = 3
    if mode == "spmv64":
        s = fa.fem_assemble(n, rho, sine)
        # the set-up tunes the CG operator's launch shape, as it does before every solve
        fa.amg_hier_destroy(fa.amg_setup(s, precision=fa.AMG_PREC_FP32))
        x = torch.randn(N, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        for it in range(reps):
            with _range(it == reps - 1):
                fa.fem_spmv(s, x, y)
        fa.fem_system_destroy(s)
    elif mode in ("vcycle32", "vcycle64"):
        s = fa.fem_assemble(n, rho, sine)
        h = fa.amg_setup(s, precision=fa.AMG_PREC_FP32 if mode == "vcycle32" else fa.AMG_PREC_FP64)
        r = torch.randn(N, dtype=torch.float64, device="cuda")
        z = torch.empty_like(r)
        for it in range(reps):
            with _range(it == reps - 1):
                fa.amg_vcycle(h, r, z)
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(s)
    elif mode == "step":
        u = torch.zeros(N, dtype=torch.float64, device="cuda")
        for it in range(reps):
            with _range(it == reps - 1):
                s = fa.fem_assemble(n, rho, sine)
                h = fa.amg_setup(s, precision=fa.AMG_PREC_FP32)
                fa.pcg_solve(s, h, None, u, tol=1e-8, use_graph=0)
                fa.amg_hier_destroy(h)
                fa.fem_system_destroy(s)
    elif mode == "galerkin":
        # the finest level's Galerkin product, recomputed from an FP32 hierarchy
        s = fa.fem_assemble(n, rho, sine)
        h = fa.amg_setup(s, precision=fa.AMG_PREC_FP32)
        for it in range(reps):
            with _range(it == reps - 1):
                fa.amg_galerkin_timed(h, 0, 1)
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(s)
    elif mode == "cgop":
        # CG's operator (double-float on the uniform grid), one timed launch per pass
        s = fa.fem_assemble(n, rho, sine)
        x = torch.randn(N, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        for it in range(reps):
            with _range(it == reps - 1):
                fa.fem_spmv_timed(s, x, y, 1)
        fa.fem_system_destroy(s)
    elif mode == "batched":
        import numpy as np
        import fem_workloads as W
        nrhs = 64
        targets, rhos = W.batched_workload(n, nrhs)
        s = fa.fem_assemble(n, 1.0 / n ** 2, W.sine_target(), keep_pencil=True)
        h = fa.amg_setup(s, precision=fa.AMG_PREC_FP32, rho_setup=float(np.max(rhos)))
        F = torch.empty((N, nrhs), dtype=torch.float64, device="cuda")
        f = torch.empty(N, dtype=torch.float64, device="cuda")
        for k, t in enumerate(targets):
            fa.fem_assemble_rhs(s, t, f)
            F[:, k] = f
        U = torch.zeros((N, nrhs), dtype=torch.float64, device="cuda")
        for it in range(reps):
            with _range(it == reps - 1):
                U.zero_()
                fa.pcg_solve(s, h, F, U, nrhs=nrhs, rho_k=rhos, tol=1e-8)
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(s)
    else:
        raise SystemExit("unknown mode " + mode)
    torch.cuda.synchronize()


if __name__ == "__main__":
    main(sys.argv)
