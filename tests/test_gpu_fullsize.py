"""Parity at the benchmark's full size: 256^3 cells (16,581,375 unknowns), rho = h^2.

The oracle cannot assemble or solve this mesh in seconds, so it computes sampled rows one
by one (from each vertex's incident tets) and the checks use properties that hold at any
size: sampled load-vector entries and operator rows, the residual of the solution on the
sampled rows, and agreement of the mixed-precision solve with an FP64 solve.
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
