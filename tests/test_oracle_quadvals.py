"""Targets given by their values at the quadrature points (the load vector of Sec. 2 for an
arbitrary ubar in L2): the oracle's load vector from per-tet point values equals the one from
the analytic target evaluated at the same points, on the Kuhn mesh (tets numbered 6 c + p:
cube c = i + n (j + n k), path p) and on a general mesh, whole-mesh and row by row.
"""
import numpy as np

import fem_workloads as W
from oracle import core


def _point_values(xyz, tets, target):
    bary, _ = core.qrule(0)
    pts = np.einsum("qa,tad->tqd", bary, xyz[np.asarray(tets)])
    return core.target_values(target, pts.reshape(-1, 3)).reshape(len(tets), 4)


def test_kuhn_quadvals_equal_the_analytic_target():
    n = 6
    xyz = W.jittered_xyz(n, 0.2, seed=3)
    for t in (W.sine_target(), W.bump_target(4)):
        vals = _point_values(xyz, core.kuhn_tets(n), t)
        s_t = core.assemble(n, t, xyz=xyz)
        s_q = core.assemble(n, {"kind": "quadvals", "values": vals}, xyz=xyz)
        assert np.max(np.abs(s_q.f - s_t.f)) <= 1e-14 * np.max(np.abs(s_t.f))
        rows = np.array([0, 7, 31, (n - 1) ** 3 - 1])
        _, _, _, f_r = core.kuhn_rows(n, {"kind": "quadvals", "values": vals}, rows, xyz=xyz)
        assert np.max(np.abs(f_r - s_t.f[rows])) <= 1e-14 * np.max(np.abs(s_t.f))


def test_general_mesh_quadvals_equal_the_analytic_target():
    x, tets, d = W.relabel_mesh(*W.bey_refine(*W.five_tet_mesh(2)), seed=1)
    t = W.bump_target(6)
    vals = _point_values(x, tets, t)
    s_t = core.assemble_mesh(x, tets, d, t)
    s_q = core.assemble_mesh(x, tets, d, {"kind": "quadvals", "values": vals})
    assert np.max(np.abs(s_q.f - s_t.f)) <= 1e-14 * np.max(np.abs(s_t.f))
    # a value moved to another point changes f: the per-tet, per-point order is used
    vals2 = vals.copy()
    vals2[:, [0, 1]] = vals2[:, [1, 0]]
    s_2 = core.assemble_mesh(x, tets, d, {"kind": "quadvals", "values": vals2})
    assert np.max(np.abs(s_2.f - s_t.f)) > 1e-6 * np.max(np.abs(s_t.f))
