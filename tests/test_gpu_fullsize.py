"""Parity at the benchmark's full size: 256^3 cells (16,581,375 unknowns), rho = h^2.

Two kinds of checks.  The oracle computes sampled rows one by one (from each vertex's
incident tets): sampled load-vector entries and operator rows, and the residual of the
solution on the sampled rows.  And the oracle assembles and solves the whole system itself
(Jacobi-PCG, its row loops on all host cores, about a minute): the GPU's solutions in every
V-cycle precision are compared with that reference vector.
"""
import numpy as np
import pytest

import fem_workloads as W
from oracle import core

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fa():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2102_03515_gb300 import build as b
    b.build()
    import paper_2102_03515_gb300 as m
    return m


def _sample_rows(m, count, seed):
    rng = np.random.default_rng(seed)
    rows = rng.integers(0, m ** 3, size=count)
    # rows touching the boundary: corners and faces of the interior grid
    edge = [0, m - 1, m * m - 1, m ** 3 - 1, (m // 2) * (1 + m + m * m)]
    return np.unique(np.concatenate([rows, edge]))


def test_full_size_rows_operator_and_solution(fa):
    n = 256
    m = n - 1
    N = m ** 3
    rho = 1.0 / n ** 2
    t = W.sine_target()
    rows = _sample_rows(m, 3000, seed=0)
    cols, K, M, f_or = core.kuhn_rows(n, t, rows)
    A_rows = rho * K + M
    valid = cols >= 0
    sys_ = fa.fem_assemble(n, rho, t)
    try:
        info = fa.fem_system_get_info(sys_)
        assert info["N"] == N and info["is_stencil"]
        f = torch.empty(N, dtype=torch.float64, device="cuda")
        fa.fem_system_get_rhs(sys_, f)
        fh = f.cpu().numpy()
        assert np.max(np.abs(fh[rows] - f_or)) <= 1e-13 * np.max(np.abs(f_or))
        # operator rows against a random vector
        x = torch.as_tensor(W.random_vector(N, 3), device="cuda")
        y = torch.empty_like(x)
        fa.fem_spmv(sys_, x, y)
        xh = x.cpu().numpy()
        xg = np.where(valid, xh[np.where(valid, cols, 0)], 0.0)
        y_or = (A_rows * xg).sum(axis=1)
        scale = (np.abs(A_rows) * np.abs(xg)).sum(axis=1)
        assert np.max(np.abs(y.cpu().numpy()[rows] - y_or) / scale) <= 1e-14
        del x, y
        # the benchmark's solve: FP32 V-cycle in FP64 flexible CG to 1e-8
        h = fa.amg_setup(sys_, precision=fa.AMG_PREC_FP32)
        u = torch.zeros(N, dtype=torch.float64, device="cuda")
        res = fa.pcg_solve(sys_, h, None, u, tol=1e-8)[0]
        fa.amg_hier_destroy(h)
        assert res["status"] == "FEM_OK" and res["relres"] <= 1e-8
        uh = u.cpu().numpy()
        ug = np.where(valid, uh[np.where(valid, cols, 0)], 0.0)
        r_rows = f_or - (A_rows * ug).sum(axis=1)
        # every residual entry is bounded by the residual norm
        assert np.max(np.abs(r_rows)) <= 1e-8 * np.linalg.norm(fh)
        # against an FP64 V-cycle solve to 1e-12
        h64 = fa.amg_setup(sys_, precision=fa.AMG_PREC_FP64)
        u64 = torch.zeros(N, dtype=torch.float64, device="cuda")
        res64 = fa.pcg_solve(sys_, h64, None, u64, tol=1e-12)[0]
        fa.amg_hier_destroy(h64)
        assert res64["status"] == "FEM_OK" and res64["relres"] <= 1e-12
        rel = (torch.linalg.norm(u - u64) / torch.linalg.norm(u64)).item()
        assert rel <= 1e-8, rel
    finally:
        fa.fem_system_destroy(sys_)


def test_full_size_solutions_match_the_oracle_reference(fa):
    # The oracle's own solution of the full system: its assembly and Jacobi-PCG to a
    # relative residual of 1e-13 (cond(D^-1 A) <= 12.2 at rho = h^2, so a few dozen
    # iterations), with the independent rows of assembly and of A x spread over the host's
    # cores.  The GPU's FP64, FP32 and BF16 V-cycle solves to 1e-13 must agree with it to
    # 1e-10; stopped at 1e-8 (the benchmark's tolerance), within cond(A) times both
    # tolerances.
    import os
    n = 256
    N = (n - 1) ** 3
    rho = 1.0 / n ** 2
    t = W.sine_target()
    core.set_threads(max(1, len(os.sched_getaffinity(0))))
    try:
        s = core.assemble(n, t)
        x_ref, it, rr = core.jacobi_pcg(s, rho, s.f, tol=1e-13)
    finally:
        core.set_threads(1)
    f_or = s.f
    del s
    assert rr <= 1e-13 and it < 200
    x_ref_d = torch.as_tensor(x_ref, device="cuda")
    nref = torch.linalg.norm(x_ref_d).item()
    sys_ = fa.fem_assemble(n, rho, t)
    try:
        f = torch.empty(N, dtype=torch.float64, device="cuda")
        fa.fem_system_get_rhs(sys_, f)
        assert np.max(np.abs(f.cpu().numpy() - f_or)) <= 1e-13 * np.max(np.abs(f_or))
        for prec in (fa.AMG_PREC_FP64, fa.AMG_PREC_FP32, fa.AMG_PREC_BF16):
            h = fa.amg_setup(sys_, precision=prec)
            try:
                for tol, bar in ((1e-13, 1e-10), (1e-8, 12.2 * 2e-8)):
                    u = torch.zeros(N, dtype=torch.float64, device="cuda")
                    res = fa.pcg_solve(sys_, h, None, u, tol=tol)[0]
                    assert res["status"] == "FEM_OK", res
                    err = (torch.linalg.norm(u - x_ref_d) / nref).item()
                    print("precision %d tol %.0e: %d iterations, |u - u_oracle| / |u_oracle| = %.3e"
                          % (prec, tol, res["iterations"], err))
                    assert err <= bar, (prec, tol, err)
            finally:
                fa.amg_hier_destroy(h)
    finally:
        fa.fem_system_destroy(sys_)
