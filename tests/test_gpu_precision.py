"""Low-precision preconditioners against the FP64 oracle.

The V-cycle may run with FP32 values and vectors, or with BF16-stored matrix values and
FP32 arithmetic, inside FP64 flexible CG (the residual, dot products, CG recurrences and
the coarsest dense solve stay FP64).  The oracle's V-cycle is FP64 throughout, so one
V-cycle is compared at a tolerance derived from the storage precision, and the solution
of a solve to 1e-13 at the FP64 parity bar.

Tolerance of one V-cycle.  Each stored value is rounded once to the storage format
(relative 2^-9 for BF16 values with round-to-nearest, 2^-24 for FP32), and the FP32
arithmetic adds 2^-24 per operation.  A V-cycle applies L stored operators in sequence
along its longest path (per level: 2 Chebyshev applications of A_l in the pre- and 2 in the
post-smoothing, 1 residual, R and P), so to first order the output moves by at most about
L u relative; with L = 8 per level over three to four levels, L u is about 6e-2 for BF16
and 2e-6 for FP32.  The errors of independent roundings do not add up in the same
direction, and the tests take 2e-2 (BF16) and 1e-6 (FP32).
"""
import numpy as np
import pytest

import fem_workloads as W
from oracle import amg, core
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

VCYCLE_TOL = {1: 1e-6, 2: 2e-2}   # AMG_PREC_FP32, AMG_PREC_BF16


@pytest.fixture(scope="module")
def fa():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2102_03515_gb300 import build as b
    b.build()
    import paper_2102_03515_gb300 as m
    return m


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("n,jit,prec", [(33, False, 1), (33, False, 2), (33, True, 1),
                                        (33, True, 2), (48, False, 2), (41, True, 2)])
def test_low_precision_vcycle_matches_oracle(fa, n, jit, prec):
    rho = 1.0 / n ** 2
    xyz = W.jittered_xyz(n, 0.2, seed=8) if jit else None
    s = core.assemble(n, W.sine_target(), xyz=xyz)
    A = s.A(rho)
    Ho = amg.build_hierarchy(A)
    sys_ = fa.fem_assemble(n, rho, W.sine_target(), xyz=xyz)
    h = fa.amg_setup(sys_, precision=prec)
    try:
        assert fa.amg_hier_get_info(h)["rows"] == [L.A.shape[0] for L in Ho]
        N = A.shape[0]
        for seed in (13, 14):
            r = W.random_vector(N, seed)
            z = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
            fa.amg_vcycle(h, _dev(r), z)
            zo = amg.vcycle(Ho, r)
            err = G.rel(z.cpu().numpy(), zo)
            assert err <= VCYCLE_TOL[prec], (n, jit, prec, err)
            # the low precision is the only difference: the error is not zero
            assert err > 1e-15
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


@pytest.mark.parametrize("n,jit,prec,tname", [(40, False, 2, "sine"), (40, True, 2, "bumps"),
                                              (40, False, 1, "box"), (33, True, 1, "sine")])
def test_low_precision_fcg_solution_matches_oracle(fa, n, jit, prec, tname):
    rho = 1.0 / n ** 2
    xyz = W.jittered_xyz(n, 0.2, seed=9) if jit else None
    t = {"sine": W.sine_target(), "box": W.box_target(0.3, 0.7), "bumps": W.bump_target(4)}[tname]
    s = core.assemble(n, t, xyz=xyz)
    x_ref, _, rr = core.jacobi_pcg(s, rho, s.f, tol=1e-14)
    sys_ = fa.fem_assemble(n, rho, t, xyz=xyz)
    h = fa.amg_setup(sys_, precision=prec)
    try:
        N = len(s.f)
        u = torch.zeros(N, dtype=torch.float64, device="cuda")
        res = fa.pcg_solve(sys_, h, None, u, tol=1e-13)[0]
        assert res["status"] == "FEM_OK", res
        assert G.rel(u.cpu().numpy(), x_ref) <= 1e-10
        # the same solve stopped at 1e-8: within cond(A) (<= 12.2 for rho = h^2) times
        # both tolerances of the reference
        u8 = torch.zeros(N, dtype=torch.float64, device="cuda")
        fa.pcg_solve(sys_, h, None, u8, tol=1e-8)
        assert G.rel(u8.cpu().numpy(), x_ref) <= 12.2 * 2e-8
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)
