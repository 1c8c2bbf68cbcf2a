"""Targets given by their values at the load vector's quadrature points (any ubar in L2,
Sec. 2) on the device, against the oracle given the same values: Kuhn meshes (uniform and
jittered, tets numbered 6 c + p) and general meshes, fem_assemble / fem_assemble_mesh /
fem_assemble_rhs; f to 1e-13 relative.  Calls that need ubar elsewhere reject them.
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


def _values(xyz, tets, target):
    bary, _ = core.qrule(0)
    pts = np.einsum("qa,tad->tqd", bary, xyz[np.asarray(tets)])
    return core.target_values(target, pts.reshape(-1, 3)).reshape(len(tets), 4)


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("n,jit", [(12, False), (11, True), (33, False)])
def test_kuhn_quadvals(fa, n, jit):
    xyz = W.jittered_xyz(n, 0.2, seed=5) if jit else None
    xyz_all = xyz if jit else W.uniform_xyz(n)
    vals = _values(xyz_all, core.kuhn_tets(n), W.bump_target(7))
    tq_or = {"kind": "quadvals", "values": vals}
    s_q = core.assemble(n, tq_or, xyz=xyz)
    tq = {"kind": "quadvals", "values": torch.as_tensor(vals, device="cuda")}
    sys_ = fa.fem_assemble(n, 1.0 / n ** 2, tq, xyz=xyz, keep_pencil=True)
    try:
        N = (n - 1) ** 3
        f = torch.empty(N, dtype=torch.float64, device="cuda")
        fa.fem_system_get_rhs(sys_, f)
        assert _rel(f.cpu().numpy(), s_q.f) <= 1e-13
        # the same values through fem_assemble_rhs, and the analytic target for comparison
        f2 = torch.empty_like(f)
        fa.fem_assemble_rhs(sys_, tq, f2)
        assert _rel(f2.cpu().numpy(), s_q.f) <= 1e-13
        s_t = core.assemble(n, W.bump_target(7), xyz=xyz)
        assert _rel(f.cpu().numpy(), s_t.f) <= 1e-13
        with pytest.raises(fa.FemError):
            fa.fem_errors(sys_, f, tq)
    finally:
        fa.fem_system_destroy(sys_)


def test_general_mesh_quadvals(fa):
    x, tets, d = W.relabel_mesh(*W.bey_refine(*W.five_tet_mesh(3)), seed=2)
    vals = _values(x, tets, W.sine_plus_one_target())
    s_q = core.assemble_mesh(x, tets, d, {"kind": "quadvals", "values": vals})
    tq = {"kind": "quadvals", "values": torch.as_tensor(vals, device="cuda")}
    sys_ = fa.fem_assemble_mesh(x, tets, d, 1e-2, tq)
    try:
        f = torch.empty(s_q.K.shape[0], dtype=torch.float64, device="cuda")
        fa.fem_system_get_rhs(sys_, f)
        assert _rel(f.cpu().numpy(), s_q.f) <= 1e-13
        with pytest.raises(fa.FemError):
            fa.fem_recover(sys_, f, tq, torch.empty_like(f), None)
        with pytest.raises(fa.FemError):
            fa.fem_error_indicator(sys_, f, tq, torch.empty(len(tets), dtype=torch.float64,
                                                             device="cuda"))
    finally:
        fa.fem_system_destroy(sys_)
