"""Run single kernels of the solver at full size, for profiler captures.

    python -m paper_2102_03515_gb300.profile_kernels spmv64 256    # FP64 stencil q = A p
    python -m paper_2102_03515_gb300.profile_kernels vcycle32 256  # one FP32 V-cycle
    python -m paper_2102_03515_gb300.profile_kernels step 256      # one assemble+setup+solve

Each mode runs its work three times (the first two as warm-up for a profiler's -s).
"""
from __future__ import annotations

import sys

import torch

from . import _binding as fa


def main(argv):
    mode = argv[1] if len(argv) > 1 else "spmv64"
    n = int(argv[2]) if len(argv) > 2 else 256
    rho = 1.0 / n ** 2
    N = (n - 1) ** 3
    sine = {"kind": "sine"}
    if mode == "spmv64":
        s = fa.fem_assemble(n, rho, sine)
        x = torch.randn(N, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        for _ in range(3):
            fa.fem_spmv(s, x, y)
        fa.fem_system_destroy(s)
    elif mode in ("vcycle32", "vcycle64"):
        s = fa.fem_assemble(n, rho, sine)
        h = fa.amg_setup(s, precision=fa.AMG_PREC_FP32 if mode == "vcycle32" else fa.AMG_PREC_FP64)
        r = torch.randn(N, dtype=torch.float64, device="cuda")
        z = torch.empty_like(r)
        for _ in range(3):
            fa.amg_vcycle(h, r, z)
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(s)
    elif mode == "step":
        u = torch.zeros(N, dtype=torch.float64, device="cuda")
        s = fa.fem_assemble(n, rho, sine)
        h = fa.amg_setup(s, precision=fa.AMG_PREC_FP32)
        fa.pcg_solve(s, h, None, u, tol=1e-8, use_graph=0)
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(s)
    else:
        raise SystemExit("unknown mode " + mode)
    torch.cuda.synchronize()


if __name__ == "__main__":
    main(sys.argv)
