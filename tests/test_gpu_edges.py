"""Edge cases of the path against the oracle: the smallest meshes (1, 8 and 27 unknowns: the
finest level is the coarsest, solved by its dense inverse), a zero right-hand side (u = 0 is
exact, no iteration), rho far on either side of h^2 (mass- and stiffness-dominated systems),
arguments outside what the library accepts (refused with FEM_EINVAL), and a general mesh
without unknowns (refused) or with a single one."""
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n", [2, 3, 4])
@pytest.mark.parametrize("fp32", [False, True])
def test_smallest_meshes_solve_like_the_oracle(fa, n, fp32):
    rho = 1e-2
    s = core.assemble(n, W.sine_target())
    x = core.cholesky_solve(s.A(rho).toarray(), s.f)
    sys_ = fa.fem_assemble(n, rho, W.sine_target())
    h = fa.amg_setup(sys_, precision=fa.AMG_PREC_FP32 if fp32 else fa.AMG_PREC_FP64)
    try:
        assert fa.amg_hier_get_info(h)["levels"] == 1
        u = torch.zeros(len(s.f), dtype=torch.float64, device="cuda")
        res = fa.pcg_solve(sys_, h, None, u, tol=1e-13)[0]
        assert res["status"] == "FEM_OK" and res["iterations"] <= 2
        assert _rel(u.cpu().numpy(), x) <= 1e-12
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


def test_zero_right_hand_side_gives_zero_without_iterating(fa):
    n = 9
    sys_ = fa.fem_assemble(n, 1e-2, W.sine_target())
    h = fa.amg_setup(sys_, precision=fa.AMG_PREC_FP32)
    try:
        N = (n - 1) ** 3
        f = torch.zeros(N, dtype=torch.float64, device="cuda")
        u = torch.full((N,), 7.0, dtype=torch.float64, device="cuda")
        res = fa.pcg_solve(sys_, h, f, u, tol=1e-8)[0]
        assert res["status"] == "FEM_OK" and res["iterations"] == 0
        assert torch.count_nonzero(u).item() == 0
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


@pytest.mark.parametrize("rho", [1e-12, 1e6])
def test_extreme_rho_solves_like_the_oracle(fa, rho):
    n = 12
    s = core.assemble(n, W.box_target(0.3, 0.7))
    x = core.cholesky_solve(s.A(rho).toarray(), s.f)
    sys_ = fa.fem_assemble(n, rho, W.box_target(0.3, 0.7))
    h = fa.amg_setup(sys_)
    try:
        u = torch.zeros(len(s.f), dtype=torch.float64, device="cuda")
        res = fa.pcg_solve(sys_, h, None, u, tol=1e-13)[0]
        assert res["status"] == "FEM_OK"
        assert _rel(u.cpu().numpy(), x) <= 1e-10
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


def test_arguments_outside_the_accepted_range_are_refused(fa):
    for n in (1, 1291):
        with pytest.raises(fa.FemError):
            fa.fem_assemble(n, 1.0, W.sine_target())
    for rho in (0.0, -1.0, float("inf")):
        with pytest.raises(fa.FemError):
            fa.fem_assemble(8, rho, W.sine_target())
    sys_ = fa.fem_assemble(8, 1.0, W.sine_target())
    try:
        with pytest.raises(fa.FemError):
            fa.amg_setup(sys_, max_row=9000)
        with pytest.raises(fa.FemError):
            fa.amg_setup(sys_, coarse_max=0)
        u = torch.zeros(7 ** 3, dtype=torch.float64, device="cuda")
        with pytest.raises(fa.FemError):
            fa.pcg_solve(sys_, None, None, u, tol=0.0)
    finally:
        fa.fem_system_destroy(sys_)


def test_a_mesh_without_unknowns_is_refused(fa):
    # one tet whose four vertices all carry the Dirichlet condition: no unknown to solve for
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    with pytest.raises(fa.FemError):
        fa.fem_assemble_mesh(xyz, tets, np.ones(4, np.uint8), 1.0, W.sine_target())
    # the same tet with one free vertex is a system of one unknown
    d = np.array([1, 1, 1, 0], np.uint8)
    s = core.assemble_mesh(xyz, tets, d, W.sine_target())
    sys_ = fa.fem_assemble_mesh(xyz, tets, d, 1.0, W.sine_target())
    try:
        assert fa.fem_system_get_info(sys_)["N"] == 1
        f = torch.empty(1, dtype=torch.float64, device="cuda")
        fa.fem_system_get_rhs(sys_, f)
        assert abs(f.item() - s.f[0]) <= 1e-13 * abs(s.f[0])
    finally:
        fa.fem_system_destroy(sys_)


def test_iteration_cap_and_cancellation(fa):
    # max_iter reached: FEM_ENOCONV with the iterate of the last iteration written; a raised
    # host cancel flag: FEM_ECANCELLED within two chunks of two iterations; a solve that
    # finishes is never reported cancelled
    import ctypes
    n = 24
    sys_ = fa.fem_assemble(n, 1.0, W.sine_target())
    h = fa.amg_setup(sys_)
    try:
        N = (n - 1) ** 3
        u = torch.zeros(N, dtype=torch.float64, device="cuda")
        res = fa.pcg_solve(sys_, h, None, u, tol=1e-14, max_iter=3)[0]
        assert res["status"] == "FEM_ENOCONV" and res["iterations"] == 3
        assert 1e-14 < res["relres"] < 1.0 and torch.count_nonzero(u).item() == N
        flag = ctypes.c_int32(1)
        with pytest.raises(fa.FemError) as ei:
            fa.pcg_solve(sys_, h, None, u, tol=1e-14, cancel_host=ctypes.pointer(flag))
        assert ei.value.status == 6   # FEM_ECANCELLED
        sys2 = fa.fem_assemble(2, 1.0, W.sine_target())   # one unknown: exact after one step
        try:
            u2 = torch.zeros(1, dtype=torch.float64, device="cuda")
            res = fa.pcg_solve(sys2, None, None, u2, tol=1e-8,
                               cancel_host=ctypes.pointer(flag))[0]
            assert res["status"] == "FEM_OK"
        finally:
            fa.fem_system_destroy(sys2)
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


def test_non_finite_right_hand_side_is_a_breakdown(fa):
    # a NaN in f (host-made failure, no GPU fault): the solve stops before its first
    # iteration with FEM_EBREAKDOWN and the iterate it started from (zero) written
    n = 12
    sys_ = fa.fem_assemble(n, 1e-2, W.sine_target())
    h = fa.amg_setup(sys_, precision=fa.AMG_PREC_FP32)
    try:
        N = (n - 1) ** 3
        f = torch.ones(N, dtype=torch.float64, device="cuda")
        f[N // 2] = float("nan")
        u = torch.full((N,), 3.0, dtype=torch.float64, device="cuda")
        with pytest.raises(fa.FemError) as ei:
            fa.pcg_solve(sys_, h, f, u, tol=1e-8)
        assert ei.value.status == 5   # FEM_EBREAKDOWN
        assert torch.count_nonzero(u).item() == 0
        f[N // 2] = float("inf")
        with pytest.raises(fa.FemError) as ei:
            fa.pcg_solve(sys_, h, f, u, tol=1e-8)
        assert ei.value.status == 5
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


def test_non_finite_slot_breaks_down_alone_in_a_batch(fa):
    # one slot of a batched session gets a NaN right-hand side: that slot reports a
    # breakdown, the other slot converges to the same result as alone
    n = 12
    rho = 1e-2
    sys_ = fa.fem_assemble(n, rho, W.sine_target(), keep_pencil=True)
    h = fa.amg_setup(sys_, precision=fa.AMG_PREC_FP32)
    b = fa.pcg_batch_create(sys_, h, 2, tol=1e-10)
    try:
        N = (n - 1) ** 3
        fgood = torch.empty(N, dtype=torch.float64, device="cuda")
        fa.fem_system_get_rhs(sys_, fgood)
        fbad = fgood.clone()
        fbad[3] = float("nan")
        s_bad = fa.pcg_batch_admit(b, fbad, rho)
        s_good = fa.pcg_batch_admit(b, fgood, rho)
        for _ in range(200):
            fa.pcg_batch_step(b, 2)
            st, it, rr = fa.pcg_batch_poll(b, 2)
            if st[s_good] != 0 and st[s_bad] != 0:
                break
        assert st[s_bad] == 2 and st[s_good] == 1
        u = torch.zeros(N, dtype=torch.float64, device="cuda")
        fa.pcg_batch_retire(b, s_good, u)
        s = core.assemble(n, W.sine_target())
        x = core.cholesky_solve(s.A(rho).toarray(), s.f)
        assert _rel(u.cpu().numpy(), x) <= 1e-8
    finally:
        fa.pcg_batch_destroy(b)
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


def test_cancel_raised_by_a_host_thread_during_a_solve(fa):
    # a long Jacobi-preconditioned solve (rho = 1 on the 96^3 mesh converges slowly, and a
    # tolerance of 1e-300 is met only once the recursive residual underflows, some 10^4
    # iterations later) runs until another host thread raises the cancel flag 0.1 s after
    # the call: FEM_ECANCELLED, with the iterations done so far in the written iterate
    import ctypes
    import threading
    import time
    n = 96
    sys_ = fa.fem_assemble(n, 1.0, W.sine_target())
    try:
        N = (n - 1) ** 3
        u = torch.zeros(N, dtype=torch.float64, device="cuda")
        flag = ctypes.c_int32(0)
        timer = threading.Timer(0.1, lambda: setattr(flag, "value", 1))
        t0 = time.time()
        timer.start()
        with pytest.raises(fa.FemError) as ei:
            fa.pcg_solve(sys_, None, None, u, tol=1e-300, max_iter=10000000,
                         cancel_host=ctypes.pointer(flag))
        timer.join()
        assert ei.value.status == 6   # FEM_ECANCELLED
        assert time.time() - t0 < 30.0
        un = u.cpu().numpy()
        assert np.all(np.isfinite(un)) and np.count_nonzero(un) == N
        # the iterate is a CG iterate: its residual is below that of the start (u = 0)
        r = torch.empty_like(u)
        fa.fem_spmv(sys_, u, r)
        f = torch.empty_like(u)
        fa.fem_system_get_rhs(sys_, f)
        assert torch.linalg.norm(f - r).item() < 1e-3 * torch.linalg.norm(f).item()
    finally:
        fa.fem_system_destroy(sys_)
