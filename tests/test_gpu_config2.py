"""The 128^3 workload (2,048,383 unknowns) in plain FP64: rho in {1, h^2, 1e-6}, the smooth
sine target and the discontinuous box (1 on (1/4, 3/4)^3), on the uniform Kuhn mesh (matrix-free
stencil) and with interior vertices jittered by up to 0.2 h (the CSR path).

The oracle computes sampled rows of K, M and f one by one from each vertex's incident tets;
the checks at this size are properties of those rows: load-vector entries and operator rows
to rounding, and the residual of the GPU solution on the sampled rows.  A solve to 1e-11
(about the attainable accuracy at rho = 1, where cond(A) is about 7e3) pins the solution to
the oracle's discrete system (u = A^-1 f up to cond(A) x 1e-11); the solve to the benchmark's
1e-8 must agree with it to cond(A) x 1e-8, and its iteration count is reported per (rho, target, mesh) to show that the
preconditioner is robust in rho.
"""
import numpy as np
import pytest

import fem_workloads as W
from oracle import core

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_CELLS = 128


@pytest.fixture(scope="module")
def fa():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2102_03515_gb300 import build as b
    b.build()
    import paper_2102_03515_gb300 as m
    return m


def _rows(m, seed):
    rng = np.random.default_rng(seed)
    rows = rng.integers(0, m ** 3, size=2000)
    edge = [0, m - 1, m * m - 1, m ** 3 - 1, (m // 2) * (1 + m + m * m)]
    return np.unique(np.concatenate([rows, edge]))


@pytest.mark.parametrize("jitter", [False, True])
@pytest.mark.parametrize("tname", ["sine", "box"])
@pytest.mark.parametrize("rho", [1.0, 1.0 / N_CELLS ** 2, 1e-6])
def test_128_fp64_amg_pcg(fa, rho, tname, jitter):
    n = N_CELLS
    m = n - 1
    N = m ** 3
    t = W.sine_target() if tname == "sine" else W.box_target()
    xyz = W.jittered_xyz(n, 0.2, seed=0) if jitter else None
    rows = _rows(m, 1 if jitter else 0)
    cols, K, M, f_or = core.kuhn_rows(n, t, rows, xyz=xyz)
    A_rows = rho * K + M
    valid = cols >= 0
    sys_ = fa.fem_assemble(n, rho, t, xyz=xyz)
    try:
        info = fa.fem_system_get_info(sys_)
        assert info["N"] == N and info["is_stencil"] == (not jitter)
        f = torch.empty(N, dtype=torch.float64, device="cuda")
        fa.fem_system_get_rhs(sys_, f)
        fh = f.cpu().numpy()
        assert np.max(np.abs(fh[rows] - f_or)) <= 1e-13 * np.max(np.abs(fh))
        x = torch.as_tensor(W.random_vector(N, 3), device="cuda")
        y = torch.empty_like(x)
        fa.fem_spmv(sys_, x, y)
        xh = x.cpu().numpy()
        xg = np.where(valid, xh[np.where(valid, cols, 0)], 0.0)
        scale = (np.abs(A_rows) * np.abs(xg)).sum(axis=1)
        assert np.max(np.abs(y.cpu().numpy()[rows] - (A_rows * xg).sum(axis=1)) / scale) <= 1e-14
        del x, y
        h = fa.amg_setup(sys_)                          # FP64 hierarchy
        u12 = torch.zeros(N, dtype=torch.float64, device="cuda")
        r12 = fa.pcg_solve(sys_, h, None, u12, tol=1e-11)[0]
        u8 = torch.zeros(N, dtype=torch.float64, device="cuda")
        r8 = fa.pcg_solve(sys_, h, None, u8, tol=1e-8)[0]
        fa.amg_hier_destroy(h)
        print("rho=%g target=%s jitter=%s: %d iterations to 1e-8, %d to 1e-11"
              % (rho, tname, jitter, r8["iterations"], r12["iterations"]))
        assert r12["status"] == "FEM_OK" and r12["relres"] <= 1e-11
        assert r8["status"] == "FEM_OK" and r8["relres"] <= 1e-8
        assert r8["iterations"] <= 60
        uh = u12.cpu().numpy()
        ug = np.where(valid, uh[np.where(valid, cols, 0)], 0.0)
        res_rows = f_or - (A_rows * ug).sum(axis=1)
        assert np.max(np.abs(res_rows)) <= 1e-11 * np.linalg.norm(fh)
        # ||u8 - u|| / ||u|| <= cond(A) * 1e-8: cond is about 7e3 at rho = 1, below 100 else
        rel = (torch.linalg.norm(u8 - u12) / torch.linalg.norm(u12)).item()
        assert rel <= (1e4 if rho == 1.0 else 1e2) * 1e-8, rel
    finally:
        fa.fem_system_destroy(sys_)
