"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: assembly and the hierarchy follow the oracle's operation order, so entries
agree to a few ulps (1e-14 relative); one V-cycle differs only by the summation order of
the fused kernels and the coarse inverse (1e-12); the solution of a solve run to a
relative residual of 1e-13 agrees with the oracle to 1e-10 (the target's parity bar).
"""
import numpy as np
import pytest

import fem_workloads as W
from oracle import amg, core
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


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


CASES = [
    # (n, rho, target, jitter, format)
    (16, 1.0 / 256, "sine", False, 0),
    (16, 1.0 / 256, "sine", False, 2),
    (12, 1.0, "box", False, 0),
    (10, 1e-6, "sine", True, 0),
    (9, 1.0 / 81, "bumps", True, 0),
]


def _target(name, seed=3):
    return {"sine": W.sine_target(), "box": W.box_target(), "bumps": W.bump_target(seed),
            "sine_plus_one": W.sine_plus_one_target()}[name]


@pytest.mark.parametrize("n,rho,tname,jit,fmt", CASES)
def test_assembly_matches_oracle(fa, n, rho, tname, jit, fmt):
    xyz = W.jittered_xyz(n, 0.2, seed=n) if jit else None
    t = _target(tname)
    s = core.assemble(n, t, xyz=xyz)
    sys_ = fa.fem_assemble(n, rho, t, xyz=xyz, fmt=fmt, keep_pencil=True)
    try:
        info = fa.fem_system_get_info(sys_)
        assert info["N"] == (n - 1) ** 3
        assert info["is_stencil"] == (not jit and fmt != 2)
        A, _ = G.export_system(fa, sys_, 0)
        K, _ = G.export_system(fa, sys_, 1)
        M, _ = G.export_system(fa, sys_, 2)
        Ao = s.A(rho)
        # same sparsity pattern, entries to a few ulps
        assert np.array_equal(A.indptr, Ao.indptr) and np.array_equal(A.indices, Ao.indices)
        assert G.sparse_rel(A, Ao) <= 1e-14
        assert G.sparse_rel(K, s.K) <= 1e-14
        assert G.sparse_rel(M, s.M) <= 1e-14
        f = torch.empty(info["N"], dtype=torch.float64, device="cuda")
        fa.fem_system_get_rhs(sys_, f)
        assert G.rel(f.cpu().numpy(), s.f) <= 1e-13
    finally:
        fa.fem_system_destroy(sys_)


@pytest.mark.parametrize("n,jit,fmt", [(16, False, 0), (16, False, 2), (48, False, 0),
                                       (33, True, 0)])
def test_operator_matches_oracle(fa, n, jit, fmt):
    rho = 1.0 / n ** 2
    xyz = W.jittered_xyz(n, 0.2, seed=1) if jit else None
    s = core.assemble(n, W.sine_target(), xyz=xyz)
    sys_ = fa.fem_assemble(n, rho, W.sine_target(), xyz=xyz, fmt=fmt)
    try:
        N = (n - 1) ** 3
        x = W.random_vector(N, 7)
        y = torch.empty(N, dtype=torch.float64, device="cuda")
        fa.fem_spmv(sys_, _dev(x), y)
        yo = core.apply(s, rho, x)
        scale = np.abs(s.A(rho)).dot(np.abs(x))
        assert np.max(np.abs(y.cpu().numpy() - yo) / scale) <= 1e-14
    finally:
        fa.fem_system_destroy(sys_)


# n = 48 and 64 (103,823 and 250,047 rows) run the Galerkin products on several thousand
# thread blocks with ragged last blocks, level 0 through the stencil's strength graph
# (uniform) or through A's CSR (jittered, format CSR)
@pytest.mark.parametrize("n,wide", [(16, False), (48, False), (33, True)])
def test_cg_operator_matches_oracle(fa, n, wide):
    # CG's operator on the uniform grid runs in double-float arithmetic (fem_spmv_timed
    # applies it as CG does).  Bound: x is rounded to 48 bits (2^-49 sum |a x|), and about a
    # dozen FP32 roundings of quantities at most 2^-23 of the row's terms stay below
    # 2^-44 sum |a_ij x_j| together.  wide: entries spread over 17 decades.
    rho = 1.0 / n ** 2
    s = core.assemble(n, W.sine_target())
    sys_ = fa.fem_assemble(n, rho, W.sine_target())
    try:
        N = (n - 1) ** 3
        x = W.random_vector(N, 17)
        if wide:
            x = x * np.exp(np.random.default_rng(5).uniform(-20.0, 20.0, N))
        y = torch.empty(N, dtype=torch.float64, device="cuda")
        ms = fa.fem_spmv_timed(sys_, _dev(x), y, 2)
        assert ms > 0.0
        yo = core.apply(s, rho, x)
        scale = np.abs(s.A(rho)).dot(np.abs(x))
        err = np.max(np.abs(y.cpu().numpy() - yo) / scale)
        assert err <= 2.0 ** -44, err
        # entries beyond the split's range: the product falls back to FP64
        x[N // 2] = 1e-30
        fa.fem_spmv_timed(sys_, _dev(x), y, 1)
        yo = core.apply(s, rho, x)
        scale = np.abs(s.A(rho)).dot(np.abs(x))
        assert np.max(np.abs(y.cpu().numpy() - yo) / scale) <= 1e-14
    finally:
        fa.fem_system_destroy(sys_)


HIER_CASES = [(16, 1.0 / 256, False, 0), (16, 1.0, False, 0), (12, 1e-6, False, 2),
              (13, 1.0 / 169, True, 0), (48, 1.0 / 48 ** 2, False, 0), (48, 1.0, True, 0),
              (64, 1.0 / 64 ** 2, False, 0), (64, 1e-6, True, 0), (48, 1e-2, False, 2)]


@pytest.mark.parametrize("n,rho,jit,fmt", HIER_CASES)
def test_hierarchy_matches_oracle(fa, n, rho, jit, fmt):
    xyz = W.jittered_xyz(n, 0.2, seed=2) if jit else None
    s = core.assemble(n, W.sine_target(), xyz=xyz)
    A = s.A(rho)
    cmax = 40 if n <= 16 else 256
    Ho = amg.build_hierarchy(A, dict(coarse_max=cmax))
    sys_ = fa.fem_assemble(n, rho, W.sine_target(), xyz=xyz, fmt=fmt)
    h = fa.amg_setup(sys_, coarse_max=cmax)
    try:
        info = fa.amg_hier_get_info(h)
        assert info["levels"] == len(Ho)
        assert info["rows"] == [L.A.shape[0] for L in Ho]
        for lev, Lo in enumerate(Ho):
            n_l = Lo.A.shape[0]
            Al = G.export_level(fa, h, lev, 0, n_l, n_l)
            assert np.array_equal(Al.indptr, Lo.A.indptr)
            assert np.array_equal(Al.indices, Lo.A.indices)
            assert G.sparse_rel(Al, Lo.A) <= 1e-13
            # entry by entry, against the size of the row's largest entry
            assert G.entrywise_rel(Al, Lo.A) <= 1e-13
            assert info["lmax"][lev] == pytest.approx(Lo.lmax, rel=1e-13)
            if Lo.coarsest:
                continue
            agg = G.export_aggregates(fa, h, lev, n_l)
            assert np.array_equal(agg, Lo.agg)  # integer work: bit-exact
            Pl = G.export_level(fa, h, lev, 1, n_l, Lo.nagg)
            Rl = G.export_level(fa, h, lev, 2, Lo.nagg, n_l)
            assert np.array_equal(Pl.indices, Lo.P.indices)
            assert G.sparse_rel(Pl, Lo.P) <= 1e-13
            assert G.sparse_rel(Rl, Lo.R) <= 1e-13
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


@pytest.mark.parametrize("n,rho,jit,smoother", [(16, 1.0 / 256, False, "chebyshev"),
                                                (16, 1.0, False, "l1"),
                                                (13, 1e-4, True, "chebyshev"),
                                                (40, 1.0 / 1600, False, "chebyshev")])
def test_vcycle_matches_oracle(fa, n, rho, jit, smoother):
    xyz = W.jittered_xyz(n, 0.2, seed=4) if jit else None
    s = core.assemble(n, W.sine_target(), xyz=xyz)
    A = s.A(rho)
    opts = dict(coarse_max=64, smoother=smoother)
    Ho = amg.build_hierarchy(A, opts)
    sys_ = fa.fem_assemble(n, rho, W.sine_target(), xyz=xyz)
    h = fa.amg_setup(sys_, coarse_max=64, smoother=1 if smoother == "l1" else 0)
    try:
        N = A.shape[0]
        r = W.random_vector(N, 11)
        z = torch.empty(N, dtype=torch.float64, device="cuda")
        fa.amg_vcycle(h, _dev(r), z)
        zo = amg.vcycle(Ho, r, opts)
        assert G.rel(z.cpu().numpy(), zo) <= 1e-12
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


@pytest.mark.parametrize("n,rho,tname,jit", [(16, 1.0 / 256, "sine", False),
                                             (16, 1.0, "box", False),
                                             (14, 1e-6, "bumps", True),
                                             (33, 1.0 / 1089, "sine", True)])
def test_pcg_solution_matches_oracle(fa, n, rho, tname, jit):
    xyz = W.jittered_xyz(n, 0.2, seed=5) if jit else None
    t = _target(tname)
    s = core.assemble(n, t, xyz=xyz)
    A = s.A(rho)
    if A.shape[0] <= 4000:
        x_ref = core.cholesky_solve(A.toarray(), s.f)
    else:
        x_ref, _, rr = core.jacobi_pcg(s, rho, s.f, tol=1e-14)
    sys_ = fa.fem_assemble(n, rho, t, xyz=xyz)
    h = fa.amg_setup(sys_)
    try:
        N = A.shape[0]
        f = torch.empty(N, dtype=torch.float64, device="cuda")
        fa.fem_system_get_rhs(sys_, f)
        for use_graph in (1, 0):
            u = torch.zeros(N, dtype=torch.float64, device="cuda")
            res = fa.pcg_solve(sys_, h, f, u, tol=1e-13, use_graph=use_graph)[0]
            assert res["status"] == "FEM_OK", res
            assert res["relres"] <= 1e-12
            assert G.rel(u.cpu().numpy(), x_ref) <= 1e-10
        # Jacobi-preconditioned CG through the same entry point
        u = torch.zeros(N, dtype=torch.float64, device="cuda")
        res = fa.pcg_solve(sys_, None, f, u, tol=1e-13, max_iter=5000)[0]
        assert res["status"] == "FEM_OK"
        assert G.rel(u.cpu().numpy(), x_ref) <= 1e-10
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


def test_pcg_is_deterministic_and_iterations_follow_oracle(fa):
    n, rho = 16, 1.0 / 256
    s = core.assemble(n, W.sine_target())
    A = s.A(rho)
    Ho = amg.build_hierarchy(A)
    xo, it_o, rr_o, _ = amg.pcg(A, s.f, lambda r: amg.vcycle(Ho, r), tol=1e-8)
    sys_ = fa.fem_assemble(n, rho, W.sine_target())
    h = fa.amg_setup(sys_)
    try:
        N = A.shape[0]
        f = _dev(s.f)
        us = []
        for _ in range(2):
            u = torch.zeros(N, dtype=torch.float64, device="cuda")
            res = fa.pcg_solve(sys_, h, f, u, tol=1e-8)[0]
            us.append(u.cpu().numpy())
            assert res["iterations"] == it_o
        assert np.array_equal(us[0], us[1])  # bitwise reproducible
        assert G.rel(us[0], xo) <= 1e-12
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)
