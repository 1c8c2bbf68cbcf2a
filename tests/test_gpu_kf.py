"""The paper's own AMG (Sec. 3.1 after KF1998) on the device: red-black coarsening,
averaging interpolation, Galerkin coarse operators and symmetric Gauss-Seidel in greedy
colour order, against the oracle's restatement.

Integer decisions (coarse/fine split, colours) are compared exactly; matrices to 1e-13
relative (the Galerkin products follow the oracle's summation order); one V-cycle to
1e-12; solutions at tol 1e-13 to 1e-10; FP32 V-cycles to 1e-5 of the FP64 one.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

import fem_workloads as W
from oracle import amg, core
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KF = {"coarsening": "kf", "smoother": "sgs", "coarse_max": 64}


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


def _gpu_opts(fa, coarsening="kf", precision=0):
    return dict(coarsening=fa.AMG_COARSEN_RED_BLACK if coarsening == "kf" else fa.AMG_COARSEN_SA,
                smoother=fa.AMG_SMOOTHER_SGS, coarse_max=64, precision=precision)


def _export_int(fa, h, level, which, n):
    a = torch.empty(n, dtype=torch.int32, device="cuda")
    fa.amg_hier_export(h, level, which, None, a, None)
    return a.cpu().numpy().astype(np.int64)


@pytest.mark.parametrize("n,rho,jit", [(12, 1.0 / 144, False), (10, 1.0, True), (13, 1e-6, False)])
def test_red_black_hierarchy_matches_oracle(fa, n, rho, jit):
    xyz = W.jittered_xyz(n, 0.2, seed=7) if jit else None
    s = core.assemble(n, W.sine_target(), xyz=xyz)
    A = s.A(rho).tocsr()
    Lo = amg.build_hierarchy(A, KF)
    sys_ = fa.fem_assemble(n, rho, W.sine_target(), xyz=xyz)
    h = fa.amg_setup(sys_, **_gpu_opts(fa))
    try:
        info = fa.amg_hier_get_info(h)
        assert info["levels"] == len(Lo)
        for lev, L in enumerate(Lo):
            N = L.A.shape[0]
            assert info["rows"][lev] == N
            Ag = G.export_level(fa, h, lev, 0, N, N)
            assert G.sparse_rel(Ag, L.A) <= 1e-13, lev
            assert np.array_equal(_export_int(fa, h, lev, 4, N), L.colours), lev
            if L.coarsest:
                continue
            cid = _export_int(fa, h, lev, 3, N)
            assert np.array_equal(cid >= 0, L.coarse), lev
            assert np.array_equal(cid[L.coarse], np.arange(L.nagg)), lev
            Nc = L.nagg
            P = G.export_level(fa, h, lev, 1, N, Nc)
            R = G.export_level(fa, h, lev, 2, Nc, N)
            assert G.sparse_rel(P, L.P) <= 1e-15 and G.sparse_rel(R, L.R) <= 1e-15, lev
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


@pytest.mark.parametrize("coarsening", ["kf", "sa"])
@pytest.mark.parametrize("n,jit", [(12, False), (9, True)])
def test_sgs_vcycle_matches_oracle(fa, coarsening, n, jit):
    rho = 1.0 / n ** 2
    xyz = W.jittered_xyz(n, 0.2, seed=8) if jit else None
    s = core.assemble(n, W.sine_target(), xyz=xyz)
    A = s.A(rho).tocsr()
    o = dict(KF, coarsening=coarsening)
    Lo = amg.build_hierarchy(A, o)
    sys_ = fa.fem_assemble(n, rho, W.sine_target(), xyz=xyz)
    h = fa.amg_setup(sys_, **_gpu_opts(fa, coarsening))
    try:
        r = W.random_vector(A.shape[0], 3)
        z = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
        fa.amg_vcycle(h, _dev(r), z)
        zo = amg.vcycle(Lo, r, o)
        assert G.rel(z.cpu().numpy(), zo) <= 1e-12
        # FP32 and BF16-valued V-cycles of the same method
        for prec, tol in ((1, 1e-5), (2, 3e-2)):
            h32 = fa.amg_setup(sys_, **_gpu_opts(fa, coarsening, precision=prec))
            z32 = torch.empty_like(z)
            fa.amg_vcycle(h32, _dev(r), z32)
            fa.amg_hier_destroy(h32)
            assert G.rel(z32.cpu().numpy(), zo) <= tol, prec
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


@pytest.mark.parametrize("n,rho", [(12, 1.0 / 144), (14, 1.0)])
def test_red_black_pcg_matches_oracle(fa, n, rho):
    s = core.assemble(n, W.sine_target())
    A = s.A(rho).tocsr()
    ref = spl.spsolve(A.tocsc(), s.f)
    Lo = amg.build_hierarchy(A, KF)
    _, it_o, _, _ = amg.pcg(A, s.f, lambda r: amg.vcycle(Lo, r, KF), tol=1e-10)
    sys_ = fa.fem_assemble(n, rho, W.sine_target())
    h = fa.amg_setup(sys_, **_gpu_opts(fa))
    try:
        u = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        res = fa.pcg_solve(sys_, h, None, u, tol=1e-10)[0]
        assert res["status"] == "FEM_OK" and res["iterations"] == it_o
        u13 = torch.zeros_like(u)
        res = fa.pcg_solve(sys_, h, None, u13, tol=1e-13)[0]
        assert G.rel(u13.cpu().numpy(), ref) <= 1e-10
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


def test_batched_rejects_gauss_seidel(fa):
    sys_ = fa.fem_assemble(8, 1.0 / 64, W.sine_target(), keep_pencil=True)
    h = fa.amg_setup(sys_, **_gpu_opts(fa))
    try:
        with pytest.raises(fa.FemError):
            fa.pcg_batch_create(sys_, h, 4)
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


@pytest.mark.parametrize("n,rho", [(16, 1.0), (17, 1.0 / 289), (12, 1e-4)])
def test_natural_order_red_black_matches_oracle(fa, n, rho):
    # visiting the unknowns in index order (the order the paper's Table 4 counts follow):
    # C/F split and colours bit-exact, Galerkin operators, and the PCG iteration count
    s = core.assemble(n, W.sine_target())
    A = s.A(rho).tocsr()
    o = dict(KF, order="natural")
    Lo = amg.build_hierarchy(A, o)
    _, it_o, _, _ = amg.pcg(A, s.f, lambda r: amg.vcycle(Lo, r, o), tol=1e-10)
    sys_ = fa.fem_assemble(n, rho, W.sine_target())
    h = fa.amg_setup(sys_, order=fa.AMG_ORDER_NATURAL, **_gpu_opts(fa))
    try:
        info = fa.amg_hier_get_info(h)
        assert info["rows"] == [L.A.shape[0] for L in Lo]
        for lev, L in enumerate(Lo):
            N = L.A.shape[0]
            Ag = G.export_level(fa, h, lev, 0, N, N)
            assert G.sparse_rel(Ag, L.A) <= 1e-13, lev
            if L.coarsest:
                continue
            cid = _export_int(fa, h, lev, 3, N)
            assert np.array_equal(cid >= 0, L.coarse), lev
        u = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        res = fa.pcg_solve(sys_, h, None, u, tol=1e-10)[0]
        assert res["status"] == "FEM_OK" and res["iterations"] == it_o
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)
