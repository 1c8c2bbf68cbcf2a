"""General tetrahedral meshes on the device (fem_assemble_mesh) against the oracle: assembly,
AMG-PCG solves with both coarsenings, batched solves, error norms and recovery.

Tolerances as for the Kuhn meshes: entries to 1e-14 relative, f to 1e-13, solutions at tol
1e-13 to 1e-10, one V-cycle to 1e-12, error norms to 1e-12.
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


MESHES = {
    "five": lambda: W.five_tet_mesh(5),
    "five_refined_relabelled": lambda: W.relabel_mesh(*W.bey_refine(*W.five_tet_mesh(3)), seed=3),
    "kuhn_jittered_refined": lambda: W.bey_refine(*W.kuhn_mesh(4, W.jittered_xyz(4, 0.2, 1))),
}


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("tname", ["sine", "bumps"])
def test_general_assembly_matches_oracle(fa, name, tname):
    xyz, tets, d = MESHES[name]()
    t = W.sine_target() if tname == "sine" else W.bump_target(5)
    rho = 1e-2
    s = core.assemble_mesh(xyz, tets, d, t)
    sys_ = fa.fem_assemble_mesh(xyz, tets, d, rho, t, keep_pencil=True)
    try:
        info = fa.fem_system_get_info(sys_)
        assert info["N"] == s.K.shape[0] and not info["is_stencil"]
        A, _ = G.export_system(fa, sys_, 0)
        K, _ = G.export_system(fa, sys_, 1)
        M, _ = G.export_system(fa, sys_, 2)
        Ao = s.A(rho)
        assert np.array_equal(A.indptr, Ao.indptr) and np.array_equal(A.indices, Ao.indices)
        assert G.sparse_rel(A, Ao) <= 1e-14
        assert G.sparse_rel(K, s.K) <= 1e-14 and G.sparse_rel(M, s.M) <= 1e-14
        f = torch.empty(info["N"], dtype=torch.float64, device="cuda")
        fa.fem_system_get_rhs(sys_, f)
        assert G.rel(f.cpu().numpy(), s.f) <= 1e-13
        f2 = torch.empty_like(f)
        fa.fem_assemble_rhs(sys_, W.bump_target(9), f2)
        so = core.assemble_mesh(xyz, tets, d, W.bump_target(9))
        assert G.rel(f2.cpu().numpy(), so.f) <= 1e-13
    finally:
        fa.fem_system_destroy(sys_)


def test_kuhn_mesh_through_the_general_path_equals_the_kuhn_path(fa):
    n, rho = 6, 1.0 / 36
    xyz = W.jittered_xyz(n, 0.2, seed=2)
    x, t, d = W.kuhn_mesh(n, xyz)
    g = fa.fem_assemble_mesh(x, t, d, rho, W.sine_target())
    k = fa.fem_assemble(n, rho, W.sine_target(), xyz=xyz)
    try:
        Ag, _ = G.export_system(fa, g, 0)
        Ak, _ = G.export_system(fa, k, 0)
        assert G.sparse_rel(Ag, Ak) <= 1e-15
        N = (n - 1) ** 3
        fg = torch.empty(N, dtype=torch.float64, device="cuda")
        fk = torch.empty_like(fg)
        fa.fem_system_get_rhs(g, fg)
        fa.fem_system_get_rhs(k, fk)
        assert G.rel(fg.cpu().numpy(), fk.cpu().numpy()) <= 1e-14
    finally:
        fa.fem_system_destroy(g)
        fa.fem_system_destroy(k)


@pytest.mark.parametrize("coarsening", ["sa", "kf"])
def test_general_mesh_solve_and_vcycle_match_oracle(fa, coarsening):
    xyz, tets, d = MESHES["five_refined_relabelled"]()
    rho = 1e-2
    s = core.assemble_mesh(xyz, tets, d, W.sine_target())
    A = s.A(rho).tocsr()
    ref = core.cholesky_solve(A.toarray(), s.f)
    o = {"coarse_max": 64}
    if coarsening == "kf":
        o.update(coarsening="kf", smoother="sgs")
    Lo = amg.build_hierarchy(A, o)
    sys_ = fa.fem_assemble_mesh(xyz, tets, d, rho, W.sine_target())
    gopt = dict(coarse_max=64)
    if coarsening == "kf":
        gopt.update(coarsening=fa.AMG_COARSEN_RED_BLACK, smoother=fa.AMG_SMOOTHER_SGS)
    h = fa.amg_setup(sys_, **gopt)
    try:
        r = W.random_vector(A.shape[0], 1)
        z = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
        fa.amg_vcycle(h, _dev(r), z)
        assert G.rel(z.cpu().numpy(), amg.vcycle(Lo, r, o)) <= 1e-12
        u = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        res = fa.pcg_solve(sys_, h, None, u, tol=1e-13)[0]
        assert res["status"] == "FEM_OK"
        assert G.rel(u.cpu().numpy(), ref) <= 1e-10
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


def test_general_mesh_batched_solve(fa):
    xyz, tets, d = MESHES["five"]()
    rhos = W.log_uniform(4, 1e-6, 1e-2, seed=2)
    s0 = core.assemble_mesh(xyz, tets, d, W.sine_target())
    N = s0.K.shape[0]
    sys_ = fa.fem_assemble_mesh(xyz, tets, d, 1e-2, W.sine_target(), keep_pencil=True)
    h = fa.amg_setup(sys_, precision=fa.AMG_PREC_FP32, coarse_max=64)
    try:
        F = torch.empty((N, 4), dtype=torch.float64, device="cuda")
        refs = []
        for k in range(4):
            t = W.bump_target(30 + k)
            f = torch.empty(N, dtype=torch.float64, device="cuda")
            fa.fem_assemble_rhs(sys_, t, f)
            F[:, k] = f
            so = core.assemble_mesh(xyz, tets, d, t)
            refs.append(core.cholesky_solve(so.A(rhos[k]).toarray(), so.f))
        U = torch.zeros((N, 4), dtype=torch.float64, device="cuda")
        res = fa.pcg_solve(sys_, h, F, U, nrhs=4, rho_k=rhos, tol=1e-11)
        for k in range(4):
            assert res[k]["status"] == "FEM_OK"
            assert G.rel(U[:, k].cpu().numpy(), refs[k]) <= 1e-9
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


def test_general_mesh_errors_and_recovery(fa):
    xyz, tets, d = MESHES["kuhn_jittered_refined"]()
    rho = 1e-2
    s = core.assemble_mesh(xyz, tets, d, W.sine_target())
    u = core.jacobi_pcg(s, rho, s.f, tol=1e-12)[0]
    scale = 1.0 / (3.0 * rho * np.pi ** 2 + 1.0)
    l2o, h1o = core.errors(s, u, {"kind": "sine_scaled", "scale": scale}, qlevel=1)
    zo, po = core.recover(s, rho, u, W.sine_target())
    sys_ = fa.fem_assemble_mesh(xyz, tets, d, rho, W.sine_target())
    try:
        r = fa.fem_errors(sys_, _dev(u), W.sine_target(), scale=scale, qlevel=1)
        assert abs(r["l2sq"] / l2o - 1) <= 1e-12 and abs(r["h1sq"] / h1o - 1) <= 1e-12
        z = torch.empty(len(u), dtype=torch.float64, device="cuda")
        p = torch.empty_like(z)
        fa.fem_recover(sys_, _dev(u), W.sine_target(), z, p)
        assert np.max(np.abs(z.cpu().numpy() - zo)) <= 1e-13 * np.max(np.abs(zo))
        assert np.max(np.abs(p.cpu().numpy() - po)) <= 1e-15 * np.max(np.abs(po))
    finally:
        fa.fem_system_destroy(sys_)


def test_invalid_meshes_are_rejected(fa):
    xyz, tets, d = W.five_tet_mesh(2)
    bad = tets.copy()
    bad[0, 0] = len(xyz) + 5
    with pytest.raises(fa.FemError):
        fa.fem_assemble_mesh(xyz, bad, d, 1.0, W.sine_target())
    flat = tets.copy()
    flat[0] = [flat[0, 0], flat[0, 0], flat[0, 1], flat[0, 2]]   # zero volume
    with pytest.raises(fa.FemError):
        fa.fem_assemble_mesh(xyz, flat, d, 1.0, W.sine_target())


def test_dof_vertex_map(fa):
    n = 7
    s = core.assemble(n, W.sine_target())
    sys_ = fa.fem_assemble(n, 1.0, W.sine_target())
    try:
        v = torch.empty(s.K.shape[0], dtype=torch.int64, device="cuda")
        fa.fem_system_dof_vertices(sys_, v)
        dof = core.interior_dof_map(n)
        expect = np.argsort(np.where(dof >= 0, dof, 10 ** 9))[: s.K.shape[0]]
        assert np.array_equal(v.cpu().numpy(), expect)
    finally:
        fa.fem_system_destroy(sys_)
    xyz, tets, d = MESHES["five_refined_relabelled"]()
    sys_ = fa.fem_assemble_mesh(xyz, tets, d, 1.0, W.sine_target())
    try:
        N = fa.fem_system_get_info(sys_)["N"]
        v = torch.empty(N, dtype=torch.int64, device="cuda")
        fa.fem_system_dof_vertices(sys_, v)
        assert np.array_equal(v.cpu().numpy(), np.flatnonzero(d == 0))
    finally:
        fa.fem_system_destroy(sys_)
