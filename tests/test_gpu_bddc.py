"""BDDC-preconditioned CG on the interface Schur complement (Sec. 3.2) against the oracle.

The solution of bddc_solve must be the discrete solution u_h = A^-1 f of the whole system
(the oracle's Cholesky or Jacobi-PCG solution): the interface CG runs to a tolerance of
1e-12 with subdomain solves to 1e-13, so the difference is bounded by cond(S_C) times those
tolerances.  The iteration count must stay bounded as rho and h change (the BDDC bound
C (1 + log(H/h))^2 does not depend on them).  A split of the slabs over two "ranks" (two host
threads on one GPU, summing through a host barrier) must give the one-process solution."""
import ctypes
import threading

import numpy as np
import pytest

import fem_workloads as W
from oracle import core
from tests import gpu_util as G

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


@pytest.mark.parametrize("n,slabs,rho,tname", [(16, 4, 1.0 / 256, "sine"), (16, 2, 1.0, "box"),
                                               (12, 3, 1e-6, "bumps"), (32, 5, 1.0 / 1024, "sine")])
def test_bddc_solution_matches_oracle(fa, n, slabs, rho, tname):
    t = {"sine": W.sine_target(), "box": W.box_target(0.3, 0.7), "bumps": W.bump_target(6)}[tname]
    s = core.assemble(n, t)
    A = s.A(rho)
    if A.shape[0] <= 4000:
        x_ref = core.cholesky_solve(A.toarray(), s.f)
    else:
        x_ref, _, _ = core.jacobi_pcg(s, rho, s.f, tol=1e-14)
    sys_ = fa.fem_assemble(n, rho, t)
    b = fa.bddc_setup(sys_, slabs, inner_tol=1e-13)
    try:
        u = torch.zeros(len(s.f), dtype=torch.float64, device="cuda")
        res = fa.bddc_solve(b, None, u, tol=1e-12, max_iter=200)
        assert res["status"] == "FEM_OK", res
        assert res["relres"] <= 1e-10
        assert G.rel(u.cpu().numpy(), x_ref) <= 1e-10
        assert res["iterations"] <= 40, res
    finally:
        fa.bddc_destroy(b)
        fa.fem_system_destroy(sys_)


def test_bddc_iterations_are_robust_in_rho(fa):
    n, slabs = 24, 4
    its = []
    for rho in (1.0, 1e-2, 1e-4, 1e-6):
        sys_ = fa.fem_assemble(n, rho, W.sine_target())
        b = fa.bddc_setup(sys_, slabs, inner_tol=1e-12)
        try:
            u = torch.zeros((n - 1) ** 3, dtype=torch.float64, device="cuda")
            res = fa.bddc_solve(b, None, u, tol=1e-8)
            assert res["status"] == "FEM_OK" and res["relres"] <= 1e-7
            its.append(res["iterations"])
        finally:
            fa.bddc_destroy(b)
            fa.fem_system_destroy(sys_)
    assert max(its) <= 30, its


class _ThreadSum:
    """All-reduce between host threads standing for ranks: every thread hands in its buffer
    at a barrier, the sum is formed once and copied back into every buffer."""

    def __init__(self, fa, ranks):
        self.fa = fa
        self.bar = threading.Barrier(ranks)
        self.views = [None] * ranks
        self.total = None

    def callback(self, rank):
        fa = self.fa

        def fn(buf, count, on_device, ctx):
            addr = ctypes.cast(buf, ctypes.c_void_p).value
            if on_device:
                v = torch.as_tensor(fa._binding._DevView(addr, count), device="cuda")
            else:
                v = torch.from_numpy(np.ctypeslib.as_array(buf, shape=(int(count),)))
            self.views[rank] = v
            self.bar.wait()
            if rank == 0:
                tot = self.views[0].clone()
                for w in self.views[1:]:
                    tot += w.to(tot.device)
                self.total = tot
            self.bar.wait()
            v.copy_(self.total.to(v.device))
            if on_device:
                torch.cuda.synchronize()
            self.bar.wait()

        return fa._binding.ALLREDUCE_FN(fn)


def test_bddc_split_over_two_ranks_matches_one_process(fa):
    n, slabs, rho = 16, 4, 1.0 / 256
    sys_ = fa.fem_assemble(n, rho, W.sine_target())
    N = (n - 1) ** 3
    b = fa.bddc_setup(sys_, slabs, inner_tol=1e-13)
    u1 = torch.zeros(N, dtype=torch.float64, device="cuda")
    r1 = fa.bddc_solve(b, None, u1, tol=1e-12)
    fa.bddc_destroy(b)
    ts = _ThreadSum(fa, 2)
    cbs = [ts.callback(0), ts.callback(1)]
    out = [None, None]
    errs = []

    def rank(r):
        try:
            bb = fa.bddc_setup(sys_, slabs, slab_begin=2 * r, slab_end=2 * r + 2, inner_tol=1e-13,
                               allreduce=cbs[r])
            u = torch.zeros(N, dtype=torch.float64, device="cuda")
            res = fa.bddc_solve(bb, None, u, allreduce=cbs[r], tol=1e-12)
            torch.cuda.synchronize()
            out[r] = (u.cpu().numpy(), res)
            fa.bddc_destroy(bb)
        except Exception as e:   # reported below
            errs.append(repr(e))
            ts.bar.abort()

    th = [threading.Thread(target=rank, args=(r,)) for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    fa.fem_system_destroy(sys_)
    assert not errs, errs
    for r in range(2):
        u, res = out[r]
        assert res["status"] == "FEM_OK" and res["iterations"] == r1["iterations"]
        assert G.rel(u, u1.cpu().numpy()) <= 1e-12
