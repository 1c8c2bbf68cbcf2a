"""General tetrahedral meshes: the generators lay out conforming meshes of the unit cube, and
the oracle's assembly on them keeps the invariants the P1 discretisation fixes (Sec. 2), is
independent of the numbering, and converges at the rate of Theorem 1.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spl

import fem_workloads as W
from oracle import core


def _meshes():
    x, t, d = W.five_tet_mesh(4)
    yield "five", x, t, d
    yield "five_refined", *W.bey_refine(x, t, d)
    yield "kuhn_refined", *W.bey_refine(*W.kuhn_mesh(3))


@pytest.mark.parametrize("name,xyz,tets,dirichlet", list(_meshes()))
def test_generated_meshes_are_conforming_partitions_of_the_cube(name, xyz, tets, dirichlet):
    det = core.tet_dets(tets, xyz)
    assert np.all(np.abs(det) > 0)
    assert abs(np.abs(det).sum() / 6.0 - 1.0) <= 1e-14
    # every face belongs to two tets, except boundary faces, which lie on the cube's surface
    faces = np.sort(np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]], tets[:, [0, 1, 3]],
                                    tets[:, [0, 1, 2]]]), axis=1)
    uf, cnt = np.unique(faces, axis=0, return_counts=True)
    assert cnt.max() == 2
    bf = uf[cnt == 1]
    on_surface = np.array([np.any(np.all((xyz[f] == 0.0) | (xyz[f] == 1.0), axis=0)) for f in bf])
    assert on_surface.all()
    surface = np.any((xyz == 0.0) | (xyz == 1.0), axis=1)
    assert np.array_equal(dirichlet.astype(bool), surface)


@pytest.mark.parametrize("name,xyz,tets,dirichlet", list(_meshes()))
def test_full_mesh_invariants(name, xyz, tets, dirichlet):
    s = core.assemble_mesh(xyz, tets, np.zeros(len(xyz), np.uint8), W.sine_target())
    one = np.ones(len(xyz))
    assert np.abs(s.K @ one).max() <= 1e-13
    assert abs(s.M.sum() - 1.0) <= 1e-14
    interior = ~dirichlet.astype(bool)
    for d in range(3):
        assert np.abs((s.K @ xyz[:, d])[interior]).max() <= 1e-13
    assert abs((s.K - s.K.T)).max() <= 1e-15 and abs((s.M - s.M.T)).max() <= 1e-15


def test_assembly_does_not_depend_on_the_numbering():
    x, t, d = W.bey_refine(*W.five_tet_mesh(3))
    s = core.assemble_mesh(x, t, d, W.bump_target(2))
    xr, tr, dr = W.relabel_mesh(x, t, d, seed=4)
    r = core.assemble_mesh(xr, tr, dr, W.bump_target(2))
    # map unknowns of the relabelled mesh back to the original ones by coordinates
    key = {tuple(p): i for i, p in enumerate(x[s.dof >= 0][np.argsort(s.dof[s.dof >= 0])])}
    xs = xr[r.dof >= 0][np.argsort(r.dof[r.dof >= 0])]
    perm = np.array([key[tuple(p)] for p in xs])
    K = s.K.toarray()[np.ix_(perm, perm)]
    assert np.abs(r.K.toarray() - K).max() <= 1e-15 * np.abs(K).max() * 10
    assert np.abs(r.f - s.f[perm]).max() <= 1e-15 * np.abs(s.f).max() * 10


def test_kuhn_generator_matches_the_structured_assembly():
    n = 4
    x, t, d = W.kuhn_mesh(n)
    g = core.assemble_mesh(x, t, d, W.sine_target())
    s = core.assemble(n, W.sine_target())
    assert np.array_equal(g.K.indptr, s.K.indptr) and np.array_equal(g.K.indices, s.K.indices)
    assert np.array_equal(g.K.data, s.K.data) and np.array_equal(g.M.data, s.M.data)
    assert np.array_equal(g.f, s.f)


def test_second_order_convergence_on_refined_unstructured_meshes():
    # Theorem 1 does not need a structured mesh: L2 error of u_rho at order 2 under refinement
    rho = 1e-2
    exact = {"kind": "sine_scaled", "scale": 1.0 / (3.0 * rho * math.pi ** 2 + 1.0)}
    mesh = W.five_tet_mesh(3)
    errs = []
    for _ in range(3):
        s = core.assemble_mesh(*mesh, W.sine_target())
        u = spl.spsolve(s.A(rho).tocsc(), s.f)
        errs.append(math.sqrt(core.errors(s, u, exact, qlevel=1)[0]))
        mesh = W.bey_refine(*mesh)
    eoc = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.7 <= e <= 2.3 for e in eoc), (errs, eoc)
