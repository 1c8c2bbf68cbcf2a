"""The adaptive loop on the device (Sec. 4.2-4.3) against the oracle: residual indicator per
tet, bulk marking, longest-edge bisection with closure, and solve -> estimate -> mark ->
refine -> assemble with the mesh kept on the device.

Bars: indicator values to 1e-12 relative per tet plus 1e-13 of the largest (all terms are
non-negative; only the face jumps of nearly affine solutions cancel); marks, thresholds, refined connectivity, vertex
coordinates and Dirichlet flags bit-exact (the refinement's decisions compare squared lengths
evaluated in the same order without contraction on both sides).
"""
import numpy as np
import pytest

import fem_workloads as W
from oracle import core
from oracle import refine as R

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


def _dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


MESHES = {
    "five_refined_relabelled": lambda: W.relabel_mesh(*W.bey_refine(*W.five_tet_mesh(3)), seed=3),
    "kuhn_jittered": lambda: W.kuhn_mesh(5, W.jittered_xyz(5, 0.2, 1)),
}


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("tname,rho,qlevel", [("box", 1e-4, 1), ("sine", 1e-2, 0),
                                              ("sine_plus_one", 1.0, 2)])
def test_indicator_matches_oracle(fa, name, tname, rho, qlevel):
    xyz, tets, d = MESHES[name]()
    # the box's faces avoid the quadrature points: on the refined five-tet mesh the paper's box
    # (0.25, 0.75)^3 puts Hammer-Stroud points exactly on its faces, where the target's value
    # (0 or 1) depends on the last bit of the point's rounding
    t = {"box": W.box_target(0.3, 0.7), "sine": W.sine_target(),
         "sine_plus_one": W.sine_plus_one_target()}[tname]
    s = core.assemble_mesh(xyz, tets, d, t)
    u = core.jacobi_pcg(s, rho, s.f, tol=1e-12)[0]
    eo = core.error_indicator(s, rho, u, t, qlevel=qlevel)
    sys_ = fa.fem_assemble_mesh(xyz, tets, d, rho, t)
    try:
        eta = torch.empty(len(tets), dtype=torch.float64, device="cuda")
        tot = fa.fem_error_indicator(sys_, _dev(u), t, eta, qlevel=qlevel)
        eg = eta.cpu().numpy()
        # a face jump of a nearly affine u_h is a difference of nearly equal gradients: its
        # rounding error scales with the gradients, so tets with tiny indicators get an
        # absolute floor of 1e-13 of the largest indicator
        err = np.abs(eg - eo)
        bound = 1e-12 * eo + 1e-13 * eo.max()
        worst = int(np.argmax(err / bound))
        assert np.all(err <= bound), (worst, eg[worst], eo[worst], eo.max())
        assert abs(tot / eo.sum() - 1.0) <= 1e-12
    finally:
        fa.fem_system_destroy(sys_)


def _marking_cases():
    for n, seed in ((1, 0), (7, 1), (1000, 2), (100_003, 3)):
        e = np.abs(W.random_vector(n, seed)) ** 3
        if n >= 1000:
            e[100:300] = e[17]                          # a block of ties
            e[400:410] = 0.0
        yield n, e


# theta = 1 only where the smallest value is not at the rounding level of the total (with
# tiny values the last decisions depend on the summation order)
@pytest.mark.parametrize("case,theta", [(c, th) for c in range(4) for th in (0.2, 0.5, 0.9)] +
                         [(0, 1.0), (1, 1.0)])
def test_bulk_marking_matches_oracle(fa, theta, case):
    n, e = list(_marking_cases())[case]
    mo = core.dorfler_mark(e, theta)
    to = e[mo].min()
    # the seeded input keeps the decision away from rounding: the sums at and just above the
    # threshold differ from theta * total by far more than a summation-order difference
    goal = theta * e.sum()
    above = e[e > to].sum()
    if theta < 1.0:
        assert e[e >= to].sum() - goal > 1e-12 * goal
    assert goal - above > 1e-12 * goal
    mark = torch.empty(n, dtype=torch.uint8, device="cuda")
    thr, nm = fa.fem_mark_bulk(_dev(e), theta, mark)
    assert np.array_equal(mark.cpu().numpy().astype(bool), mo)
    assert thr == to and nm == mo.sum()


def test_bulk_marking_edge_cases(fa):
    mark = torch.empty(5, dtype=torch.uint8, device="cuda")
    thr, nm = fa.fem_mark_bulk(_dev(np.zeros(5)), 0.5, mark)
    assert nm == 0 and not mark.any()
    assert not core.dorfler_mark(np.zeros(5), 0.5).any()
    for bad in (np.array([1.0, -1.0, 2.0, 0.0, 1.0]), np.array([1.0, np.nan, 2.0, 0.0, 1.0]),
                np.array([1.0, np.inf, 2.0, 0.0, 1.0])):
        with pytest.raises(fa.FemError):
            fa.fem_mark_bulk(_dev(bad), 0.5, mark)
    with pytest.raises(fa.FemError):
        fa.fem_mark_bulk(_dev(np.ones(5)), 0.0, mark)


REFINE_MESHES = {
    "kuhn4": lambda: W.kuhn_mesh(4),
    "kuhn4_jittered": lambda: W.kuhn_mesh(4, W.jittered_xyz(4, 0.25, 5)),
    "five4": lambda: W.five_tet_mesh(4),
    "five3_relabelled_refined": lambda: W.relabel_mesh(*W.bey_refine(*W.five_tet_mesh(3)), seed=8),
}


@pytest.mark.parametrize("name", list(REFINE_MESHES))
def test_refinement_matches_oracle(fa, name):
    xyz, tets, d = REFINE_MESHES[name]()
    m = fa.fem_mesh_create(xyz, tets, d)
    try:
        rng = np.random.default_rng(21)
        for frac in (0.1, 0.3, 0.02, 0.0):
            marked = rng.random(len(tets)) < frac
            xo, to, do, po = R.refine(xyz, tets, d, marked)
            st = fa.fem_mesh_refine(m, _dev(marked, torch.uint8))
            xg, tg, dg = fa.fem_mesh_download(m)
            assert st["passes"] == po
            assert st["new_tets"] == len(to) - len(tets)
            assert np.array_equal(tg, to)
            assert np.array_equal(xg.view(np.uint64), xo.view(np.uint64))
            assert np.array_equal(dg, do)
            xyz, tets, d = xo, to, do
    finally:
        fa.fem_mesh_destroy(m)


def test_adaptive_loop_stays_on_the_device(fa):
    # box target (Sec. 4.2): refine where the discontinuity sits; properties that hold at any
    # size: conforming, volume kept, Dirichlet flags on the cube's surface, the estimate falls
    rho = 1e-4
    t = W.box_target()
    m = fa.fem_mesh_create(*W.kuhn_mesh(6))
    totals = []
    try:
        for it in range(6):
            sys_ = fa.fem_assemble_on_mesh(m, rho, t)
            h = fa.amg_setup(sys_, coarse_max=64)
            info = fa.fem_system_get_info(sys_)
            nt = fa.fem_mesh_get_info(m)["nt"]
            u = torch.zeros(info["N"], dtype=torch.float64, device="cuda")
            res = fa.pcg_solve(sys_, h, None, u, tol=1e-10)[0]
            assert res["status"] == "FEM_OK"
            eta = torch.empty(nt, dtype=torch.float64, device="cuda")
            totals.append(fa.fem_error_indicator(sys_, u, t, eta))
            mark = torch.empty(nt, dtype=torch.uint8, device="cuda")
            _, nm = fa.fem_mark_bulk(eta, 0.5, mark)
            assert nm >= 1
            fa.amg_hier_destroy(h)
            fa.fem_system_destroy(sys_)
            fa.fem_mesh_refine(m, mark)
        xyz, tets, d = fa.fem_mesh_download(m)
        faces = np.sort(np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]],
                                        tets[:, [0, 1, 3]], tets[:, [0, 1, 2]]]), axis=1)
        _, cnt = np.unique(faces, axis=0, return_counts=True)
        assert cnt.max() == 2
        assert abs(np.abs(core.tet_dets(tets, xyz)).sum() / 6.0 - 1.0) <= 1e-13
        assert np.array_equal(d, W._cube_boundary(xyz))
        assert len(tets) > 3 * 6 * 6 ** 3
        assert totals[-1] < totals[0]
    finally:
        fa.fem_mesh_destroy(m)


def test_invalid_inputs_are_rejected(fa):
    # indicator on a Kuhn-mesh system
    k = fa.fem_assemble(6, 1e-2, W.sine_target())
    try:
        with pytest.raises(fa.FemError):
            fa.fem_error_indicator(k, torch.zeros(125, dtype=torch.float64, device="cuda"),
                                   W.sine_target(), torch.empty(1296, dtype=torch.float64,
                                                                device="cuda"))
    finally:
        fa.fem_system_destroy(k)
    # three tets on one face
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0, 0, -1], [0.3, 0.3, 0.9]],
                   dtype=np.float64)
    tets = np.array([[0, 1, 2, 3], [0, 2, 1, 4], [0, 1, 2, 5]], dtype=np.int32)
    with pytest.raises(fa.FemError):
        fa.fem_mesh_create(xyz, tets, np.ones(6, np.uint8))
    # zero volume
    x, t, d = W.five_tet_mesh(2)
    flat = t.copy()
    flat[0] = [flat[0, 0], flat[0, 0], flat[0, 1], flat[0, 2]]
    with pytest.raises(fa.FemError):
        fa.fem_mesh_create(x, flat, d)


def _graded_box_mesh(n0=6, fac=0.7, steps=12):
    """Kuhn mesh refined by longest-edge bisection towards the faces of the box (0.25, 0.75)^3
    (tets whose centroid lies within 0.2 fac^k of the box's surface at step k): a mesh
    graded like the adaptive meshes of the discontinuous target."""
    x, t, d = W.kuhn_mesh(n0)
    for k in range(steps):
        c = x[t].mean(axis=1)
        inside = np.all((c > 0.25) & (c < 0.75), axis=1)
        d_in = np.min(np.minimum(c - 0.25, 0.75 - c), axis=1)
        d_out = np.linalg.norm(np.maximum(np.maximum(0.25 - c, c - 0.75), 0.0), axis=1)
        x, t, d, _ = R.refine(x, t, d, np.where(inside, d_in, d_out) < 0.2 * fac ** k)
    return x, t, d


def test_graded_mesh_hierarchy_with_long_coarse_rows(fa):
    # 44K unknowns; the first coarse operator has rows of about 700 entries, more than the
    # shared-memory product tables hold, so its Galerkin product takes the long-row path
    from oracle import amg
    from tests import gpu_util as G
    xyz, tets, d = _graded_box_mesh()
    rho = 1e-6
    s = core.assemble_mesh(xyz, tets, d, W.box_target())
    A = s.A(rho).tocsr()
    Ho = amg.build_hierarchy(A)
    assert max(np.diff(L.A.indptr).max() for L in Ho) > 512
    sys_ = fa.fem_assemble_mesh(xyz, tets, d, rho, W.box_target())
    h = fa.amg_setup(sys_)
    try:
        info = fa.amg_hier_get_info(h)
        assert info["levels"] == len(Ho)
        for lev, Lo in enumerate(Ho):
            n_l = Lo.A.shape[0]
            Al = G.export_level(fa, h, lev, 0, n_l, n_l)
            assert np.array_equal(Al.indptr, Lo.A.indptr), lev
            assert np.array_equal(Al.indices, Lo.A.indices), lev
            assert G.sparse_rel(Al, Lo.A) <= 1e-13, lev
            if Lo.coarsest:
                continue
            assert np.array_equal(G.export_aggregates(fa, h, lev, n_l), Lo.agg), lev
            Rl = G.export_level(fa, h, lev, 2, Lo.nagg, n_l)
            assert G.sparse_rel(Rl, Lo.R) <= 1e-13, lev
        r = W.random_vector(A.shape[0], 5)
        z = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
        fa.amg_vcycle(h, _dev(r), z)
        assert G.rel(z.cpu().numpy(), amg.vcycle(Ho, r, {})) <= 1e-12
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


@pytest.mark.parametrize("max_row", [500, 300])
def test_row_limit_makes_the_dense_level_the_coarsest(fa, max_row):
    # on the graded mesh the first coarse operator has rows of about 700 entries and the
    # restriction rows of about 360: a limit of 500 stops at the Galerkin product, 300 at the
    # restriction; either way level 0 is the coarsest and the V-cycle is its smoother alone
    from oracle import amg
    from tests import gpu_util as G
    xyz, tets, d = _graded_box_mesh()
    rho = 1e-6
    s = core.assemble_mesh(xyz, tets, d, W.box_target())
    A = s.A(rho).tocsr()
    Ho = amg.build_hierarchy(A, {"max_row": max_row})
    assert len(Ho) == 1 and Ho[0].coarsest and Ho[0].Ainv is None
    sys_ = fa.fem_assemble_mesh(xyz, tets, d, rho, W.box_target())
    h = fa.amg_setup(sys_, max_row=max_row)
    try:
        assert fa.amg_hier_get_info(h)["levels"] == 1
        r = W.random_vector(A.shape[0], 6)
        z = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
        fa.amg_vcycle(h, _dev(r), z)
        assert G.rel(z.cpu().numpy(), amg.vcycle(Ho, r, {})) <= 1e-12
        u = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        res = fa.pcg_solve(sys_, h, None, u, tol=1e-8)[0]
        assert res["status"] == "FEM_OK"
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)
