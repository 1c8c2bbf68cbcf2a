"""Batched multi-vector PCG (many targets and rho values on one mesh) against the oracle.

Each column is an independent solve of (rho_k K + M) u_k = f_k; the batched path uses an
FP32 V-cycle inside FP64 flexible CG, so a column solved to ||r|| / ||f|| <= 1e-11 agrees
with the oracle's exact solution to 1e-9 relative.  On the uniform grid CG's operator runs
in double-float arithmetic for tolerances down to 1e-12 and in FP64 below: a solve to 1e-13
(FP64 operator) agrees with the oracle to 1e-11.  A slot's result must not depend on the
other slots in the batch: compared bitwise.
"""
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


def _setup(fa, n, jit=False, precision=1):
    xyz = W.jittered_xyz(n, 0.2, seed=9) if jit else None
    rho_ref = 1.0 / n ** 2
    sys_ = fa.fem_assemble(n, rho_ref, W.sine_target(), xyz=xyz, keep_pencil=True)
    h = fa.amg_setup(sys_, precision=precision, coarse_max=64)
    return sys_, h, xyz


@pytest.mark.parametrize("n,jit,nrhs", [(12, False, 8), (11, True, 5), (16, False, 3)])
def test_batched_solve_matches_oracle(fa, n, jit, nrhs):
    sys_, h, xyz = _setup(fa, n, jit)
    try:
        N = (n - 1) ** 3
        targets = [W.bump_target(1000 + k) for k in range(nrhs)]
        rhos = W.log_uniform(nrhs, 1e-6, 1e-2, seed=5)
        F = torch.empty((N, nrhs), dtype=torch.float64, device="cuda")
        refs = []
        for k, t in enumerate(targets):
            f = torch.empty(N, dtype=torch.float64, device="cuda")
            fa.fem_assemble_rhs(sys_, t, f)
            s = core.assemble(n, t, xyz=xyz)
            assert G.rel(f.cpu().numpy(), s.f) <= 1e-13
            F[:, k] = f
            A = s.A(rhos[k]).toarray()
            refs.append(core.cholesky_solve(A, s.f))
        U = torch.zeros((N, nrhs), dtype=torch.float64, device="cuda")
        res = fa.pcg_solve(sys_, h, F.contiguous(), U, nrhs=nrhs, rho_k=rhos, tol=1e-11)
        Uh = U.cpu().numpy()
        for k in range(nrhs):
            assert res[k]["status"] == "FEM_OK", res[k]
            assert res[k]["relres"] <= 1e-10
            assert G.rel(Uh[:, k], refs[k]) <= 1e-9, k
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


@pytest.mark.parametrize("n,nrhs", [(12, 4), (16, 3)])
def test_batched_solve_fp64_operator_matches_oracle(fa, n, nrhs):
    sys_, h, xyz = _setup(fa, n)
    try:
        N = (n - 1) ** 3
        rhos = W.log_uniform(nrhs, 1e-6, 1e-2, seed=7)
        F = torch.empty((N, nrhs), dtype=torch.float64, device="cuda")
        refs = []
        for k in range(nrhs):
            t = W.bump_target(2000 + k)
            f = torch.empty(N, dtype=torch.float64, device="cuda")
            fa.fem_assemble_rhs(sys_, t, f)
            s = core.assemble(n, t)
            F[:, k] = f
            refs.append(core.cholesky_solve(s.A(rhos[k]).toarray(), s.f))
        U = torch.zeros((N, nrhs), dtype=torch.float64, device="cuda")
        res = fa.pcg_solve(sys_, h, F.contiguous(), U, nrhs=nrhs, rho_k=rhos, tol=1e-13)
        Uh = U.cpu().numpy()
        for k in range(nrhs):
            assert res[k]["status"] == "FEM_OK", res[k]
            assert res[k]["relres"] <= 1e-12
            assert G.rel(Uh[:, k], refs[k]) <= 1e-11, k
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


def _run_session(fa, sys_, h, slots, plan, N):
    """plan: list of (step_before_admit, f, rho); returns the solution of the first entry."""
    b = fa.pcg_batch_create(sys_, h, slots, tol=1e-10, max_iter=200)
    try:
        first_slot = None
        for k, (wait, f, rho) in enumerate(plan):
            if wait:
                fa.pcg_batch_step(b, wait)
            slot = fa.pcg_batch_admit(b, f, rho)
            if k == 0:
                first_slot = slot
        for _ in range(100):
            fa.pcg_batch_step(b, 4)
            st, it, rr = fa.pcg_batch_poll(b, slots)
            if st[first_slot] != 0:
                break
        assert st[first_slot] == 1, (st, it, rr)
        u = torch.empty(N, dtype=torch.float64, device="cuda")
        fa.pcg_batch_retire(b, first_slot, u)
        return u.cpu().numpy(), first_slot, int(it[first_slot])
    finally:
        fa.pcg_batch_destroy(b)


def test_slot_result_is_the_same_alone_and_in_the_mix(fa):
    n = 13
    sys_, h, _ = _setup(fa, n)
    try:
        N = (n - 1) ** 3
        fs = []
        for k in range(6):
            f = torch.empty(N, dtype=torch.float64, device="cuda")
            fa.fem_assemble_rhs(sys_, W.bump_target(50 + k), f)
            fs.append(f)
        rhos = [3e-3, 1e-6, 2e-4, 5e-5, 1e-2, 7e-6]
        alone, s0, it0 = _run_session(fa, sys_, h, 8, [(0, fs[0], rhos[0])], N)
        # the same request admitted third, two iterations after the others started
        mix_plan = [(0, fs[1], rhos[1]), (0, fs[2], rhos[2])]
        mix_plan = [(2, fs[0], rhos[0])] + mix_plan  # first entry is the request under test
        # admit the others first, then the request: reorder so the request joins late
        b = fa.pcg_batch_create(sys_, h, 8, tol=1e-10, max_iter=200)
        try:
            for f, r in zip(fs[1:], rhos[1:]):
                fa.pcg_batch_admit(b, f, r)
            fa.pcg_batch_step(b, 3)
            slot = fa.pcg_batch_admit(b, fs[0], rhos[0])
            assert slot == 5
            for _ in range(100):
                fa.pcg_batch_step(b, 2)
                st, it, rr = fa.pcg_batch_poll(b, 8)
                if st[slot] != 0:
                    break
            assert st[slot] == 1
            u = torch.empty(N, dtype=torch.float64, device="cuda")
            fa.pcg_batch_retire(b, slot, u)
            mixed = u.cpu().numpy()
            assert int(it[slot]) == it0
        finally:
            fa.pcg_batch_destroy(b)
        assert np.array_equal(alone, mixed)
        del mix_plan, s0
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


def test_admission_limits_and_footprint(fa):
    n = 9
    sys_, h, _ = _setup(fa, n)
    try:
        N = (n - 1) ** 3
        f = torch.empty(N, dtype=torch.float64, device="cuda")
        fa.fem_assemble_rhs(sys_, W.bump_target(3), f)
        f1 = fa.pcg_batch_footprint(sys_, h, 1)
        f8 = fa.pcg_batch_footprint(sys_, h, 8)
        assert 0 < f1 < f8
        b = fa.pcg_batch_create(sys_, h, 2)
        try:
            s0 = fa.pcg_batch_admit(b, f, 1e-3)
            s1 = fa.pcg_batch_admit(b, f, 1e-4)
            assert {s0, s1} == {0, 1}
            with pytest.raises(fa.FemError) as ei:
                fa.pcg_batch_admit(b, f, 1e-5)
            assert ei.value.status == 2  # FEM_ENOMEM: no free slot
            u = torch.empty(N, dtype=torch.float64, device="cuda")
            fa.pcg_batch_step(b, 30)
            fa.pcg_batch_retire(b, s0, u)
            assert fa.pcg_batch_admit(b, f, 1e-5) == s0
            with pytest.raises(fa.FemError):
                fa.pcg_batch_admit(b, f, -1.0)
        finally:
            fa.pcg_batch_destroy(b)
        # a batch needs the pencil
        plain = fa.fem_assemble(n, 1.0 / n ** 2, W.sine_target())
        hp = fa.amg_setup(plain)
        with pytest.raises(fa.FemError):
            fa.pcg_batch_create(plain, hp, 2)
        fa.amg_hier_destroy(hp)
        fa.fem_system_destroy(plain)
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)
