"""ctypes wrapper of the oracle's C core (``oracle/oracle.c``).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Numbering (shared convention, not shared code): vertex (i, j, k) of the
(n+1)^3 grid has index ``i + (n+1)*(j + (n+1)*k)``; the interior vertex
(i, j, k), 1 <= i, j, k <= n-1, is unknown number
``(i-1) + (n-1)*((j-1) + (n-1)*(k-1))``.  Boundary vertices carry the
homogeneous Dirichlet value 0 and are not unknowns (Sec. 2: V_h = S_h^1 cap H_0^1).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

T_SINE, T_BOX, T_BUMPS, T_SINE_PLUS_ONE, T_SINE_SCALED, T_QUADVALS = 0, 1, 2, 3, 4, 5
_KINDS = {"sine": T_SINE, "box": T_BOX, "bumps": T_BUMPS,
          "sine_plus_one": T_SINE_PLUS_ONE, "sine_scaled": T_SINE_SCALED,
          "quadvals": T_QUADVALS}


def build(force: bool = False) -> str:
    """Compile the C core with gcc (no FMA contraction: same results on x86 and Arm), with
    OpenMP where gcc has it (row loops only; the results do not depend on the threads)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                "-o", tmp, _SRC, "-lm"]
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True)
        if r.returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


class _Target(C.Structure):
    _fields_ = [("kind", C.c_int), ("nb", C.c_int), ("c", C.POINTER(C.c_double)),
                ("w", C.POINTER(C.c_double)), ("a", C.POINTER(C.c_double)),
                ("lo", C.c_double), ("hi", C.c_double), ("scale", C.c_double),
                ("qv", C.POINTER(C.c_double))]


class _Sys(C.Structure):
    _fields_ = [("nrows", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.POINTER(C.c_int64)),
                ("col", C.POINTER(C.c_int32)), ("K", C.POINTER(C.c_double)),
                ("M", C.POINTER(C.c_double)), ("f", C.POINTER(C.c_double))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER
            lib.ora_set_threads.argtypes = [C.c_int]
            lib.ora_set_threads.restype = C.c_int
            lib.ora_set_threads(1)
            lib.ora_uniform_xyz.argtypes = [C.c_int, P(C.c_double)]
            lib.ora_kuhn_tets.argtypes = [C.c_int, P(C.c_int32)]
            lib.ora_element.argtypes = [P(C.c_double), P(C.c_double), P(C.c_double)]
            lib.ora_element.restype = C.c_double
            lib.ora_qrule.argtypes = [C.c_int, P(C.c_double), P(C.c_double)]
            lib.ora_qrule.restype = C.c_int
            lib.ora_assemble.argtypes = [C.c_int64, P(C.c_double), C.c_int64, P(C.c_int32),
                                         P(C.c_int32), C.c_int64, P(_Target), C.c_int, P(_Sys)]
            lib.ora_assemble.restype = C.c_int
            lib.ora_sys_free.argtypes = [P(_Sys)]
            lib.ora_tet_dets.argtypes = [C.c_int64, P(C.c_int32), P(C.c_double), P(C.c_double)]
            lib.ora_apply.argtypes = [P(_Sys), C.c_double, P(C.c_double), P(C.c_double)]
            lib.ora_jacobi_pcg.argtypes = [P(_Sys), C.c_double, P(C.c_double), P(C.c_double),
                                           C.c_double, C.c_int, P(C.c_double)]
            lib.ora_jacobi_pcg.restype = C.c_int
            lib.ora_cholesky.argtypes = [C.c_int, P(C.c_double)]
            lib.ora_cholesky.restype = C.c_int
            lib.ora_cholesky_solve.argtypes = [C.c_int, P(C.c_double), P(C.c_double),
                                               P(C.c_double)]
            lib.ora_kuhn_rows.argtypes = [C.c_int, P(C.c_double), P(_Target), C.c_int,
                                          C.c_int64, P(C.c_int64), P(C.c_int32),
                                          P(C.c_double), P(C.c_double), P(C.c_double)]
            lib.ora_kuhn_rows.restype = C.c_int
            lib.ora_target_values.argtypes = [P(_Target), C.c_int64, P(C.c_double),
                                              P(C.c_double)]
            lib.ora_errors.argtypes = [C.c_int64, P(C.c_double), C.c_int64, P(C.c_int32),
                                       P(C.c_double), P(_Target), C.c_int, P(C.c_double),
                                       P(C.c_double)]
            _lib = lib
    return _lib


def set_threads(n: int) -> int:
    """Threads for the C core's row loops (assembly, A x); 1 (serial) unless set.  Returns
    the count in effect (1 when the core was built without OpenMP)."""
    return int(_load().ora_set_threads(int(n)))


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


# ---------------------------------------------------------------- mesh

def uniform_xyz(n: int) -> np.ndarray:
    xyz = np.empty(((n + 1) ** 3, 3), dtype=np.float64)
    _load().ora_uniform_xyz(n, _dp(xyz))
    return xyz


def kuhn_tets(n: int) -> np.ndarray:
    tets = np.empty((6 * n ** 3, 4), dtype=np.int32)
    _load().ora_kuhn_tets(n, _ip(tets))
    return tets


def interior_dof_map(n: int) -> np.ndarray:
    """vertex -> unknown index (or -1 on the boundary)."""
    i = np.arange(n + 1)
    K, J, I = np.meshgrid(i, i, i, indexing="ij")
    inside = (I > 0) & (I < n) & (J > 0) & (J < n) & (K > 0) & (K < n)
    d = (I - 1) + (n - 1) * ((J - 1) + (n - 1) * (K - 1))
    return np.where(inside, d, -1).astype(np.int32).reshape(-1)


def element(X: np.ndarray):
    """(det J, K_e, M_e) of one tet with vertex coordinates X (4x3)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    Ke = np.empty((4, 4)); Me = np.empty((4, 4))
    det = _load().ora_element(_dp(X), _dp(Ke), _dp(Me))
    return det, Ke, Me


def qrule(level: int):
    npts = 4 * 8 ** level
    bary = np.empty((npts, 4)); wt = np.empty(npts)
    _load().ora_qrule(level, _dp(bary), _dp(wt))
    return bary, wt


def tet_dets(tets: np.ndarray, xyz: np.ndarray) -> np.ndarray:
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    out = np.empty(len(tets))
    _load().ora_tet_dets(len(tets), _ip(tets), _dp(xyz), _dp(out))
    return out


# ---------------------------------------------------------------- targets

def _target_struct(target: dict):
    kind = _KINDS[target["kind"]]
    keep = []
    t = _Target()
    t.kind = kind
    t.nb = 0
    t.lo = float(target.get("lo", 0.25))
    t.hi = float(target.get("hi", 0.75))
    t.scale = float(target.get("scale", 1.0))
    if kind == T_QUADVALS:
        # ubar at the 4 points of the degree-2 rule of every tet, [tet][point]
        q = np.ascontiguousarray(target["values"], dtype=np.float64).reshape(-1)
        keep.append(q)
        t.qv = _dp(q)
    if kind == T_BUMPS:
        c = np.ascontiguousarray(target["centers"], dtype=np.float64).reshape(-1, 3)
        w = np.ascontiguousarray(target["widths"], dtype=np.float64).reshape(-1)
        a = np.ascontiguousarray(target["amps"], dtype=np.float64).reshape(-1)
        keep += [c, w, a]
        t.nb = len(w)
        t.c, t.w, t.a = _dp(c), _dp(w), _dp(a)
    return t, keep


# ---------------------------------------------------------------- assembly

class System:
    """Assembled K, M (scipy CSR, sorted columns) and load f on the unknowns."""

    def __init__(self, K, M, f, dof, n, xyz, tets):
        self.K, self.M, self.f, self.dof, self.n = K, M, f, dof, n
        self.xyz, self.tets = xyz, tets

    def A(self, rho: float):
        """A = rho K + M (Sec. 2, eq. (linsys)); same pattern as K and M."""
        return sp.csr_matrix((rho * self.K.data + self.M.data, self.K.indices, self.K.indptr),
                             shape=self.K.shape)

    def full_vector(self, u: np.ndarray) -> np.ndarray:
        """Extend an unknown vector by the Dirichlet zeros to all vertices."""
        U = np.zeros(len(self.dof))
        m = self.dof >= 0
        U[m] = u[self.dof[m]]
        return U


def assemble(n: int, target: dict, xyz: np.ndarray | None = None, qlevel: int = 0,
             full: bool = False) -> System:
    """Assemble the P1 system on the Kuhn mesh of the unit cube with n cells per side.

    ``xyz`` overrides the vertex coordinates (e.g. a jittered mesh); ``full``
    keeps every vertex as an unknown (no Dirichlet elimination; used by the
    invariant checks)."""
    lib = _load()
    if xyz is None:
        xyz = uniform_xyz(n)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = kuhn_tets(n)
    nv = (n + 1) ** 3
    dof = np.arange(nv, dtype=np.int32) if full else interior_dof_map(n)
    ndof = int((dof >= 0).sum())
    t, keep = _target_struct(target)
    s = _Sys()
    rc = lib.ora_assemble(nv, _dp(xyz), len(tets), _ip(tets), _ip(dof), ndof, C.byref(t),
                          qlevel, C.byref(s))
    if rc == -1:
        raise MemoryError("oracle assembly: allocation failed")
    try:
        if rc == -2:
            raise ValueError("oracle assembly: degenerate tetrahedron")
        if rc == -3:
            raise ValueError("oracle assembly: per-tet target values need the 4-point rule")
        nnz = s.nnz
        rowptr = np.ctypeslib.as_array(s.rowptr, (ndof + 1,)).copy()
        col = np.ctypeslib.as_array(s.col, (nnz,)).copy() if nnz else np.zeros(0, np.int32)
        Kv = np.ctypeslib.as_array(s.K, (nnz,)).copy() if nnz else np.zeros(0)
        Mv = np.ctypeslib.as_array(s.M, (nnz,)).copy() if nnz else np.zeros(0)
        f = np.ctypeslib.as_array(s.f, (ndof,)).copy() if ndof else np.zeros(0)
    finally:
        lib.ora_sys_free(C.byref(s))
    K = sp.csr_matrix((Kv, col, rowptr), shape=(ndof, ndof))
    M = sp.csr_matrix((Mv, col.copy(), rowptr.copy()), shape=(ndof, ndof))
    K.has_sorted_indices = True
    M.has_sorted_indices = True
    return System(K, M, f, dof, n, xyz, tets)


def assemble_mesh(xyz: np.ndarray, tets: np.ndarray, dirichlet: np.ndarray, target: dict,
                  qlevel: int = 0) -> System:
    """Assemble on a general tetrahedral mesh; the unknowns are the vertices not flagged in
    ``dirichlet``, numbered in increasing vertex order."""
    lib = _load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    tets = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    free = np.asarray(dirichlet) == 0
    dof = np.full(len(xyz), -1, dtype=np.int32)
    dof[free] = np.arange(int(free.sum()), dtype=np.int32)
    ndof = int(free.sum())
    t, keep = _target_struct(target)
    s = _Sys()
    rc = lib.ora_assemble(len(xyz), _dp(xyz), len(tets), _ip(tets), _ip(dof), ndof, C.byref(t),
                          qlevel, C.byref(s))
    if rc == -1:
        raise MemoryError("oracle assembly: allocation failed")
    try:
        if rc == -2:
            raise ValueError("oracle assembly: degenerate tetrahedron")
        if rc == -3:
            raise ValueError("oracle assembly: per-tet target values need the 4-point rule")
        nnz = s.nnz
        rowptr = np.ctypeslib.as_array(s.rowptr, (ndof + 1,)).copy()
        col = np.ctypeslib.as_array(s.col, (nnz,)).copy()
        Kv = np.ctypeslib.as_array(s.K, (nnz,)).copy()
        Mv = np.ctypeslib.as_array(s.M, (nnz,)).copy()
        f = np.ctypeslib.as_array(s.f, (ndof,)).copy()
    finally:
        lib.ora_sys_free(C.byref(s))
    K = sp.csr_matrix((Kv, col, rowptr), shape=(ndof, ndof))
    M = sp.csr_matrix((Mv, col.copy(), rowptr.copy()), shape=(ndof, ndof))
    K.has_sorted_indices = True
    M.has_sorted_indices = True
    return System(K, M, f, dof, None, xyz, tets)


def _sys_struct(system: System):
    K = system.K
    rowptr = np.ascontiguousarray(K.indptr, dtype=np.int64)
    col = np.ascontiguousarray(K.indices, dtype=np.int32)
    Kv = np.ascontiguousarray(K.data, dtype=np.float64)
    Mv = np.ascontiguousarray(system.M.data, dtype=np.float64)
    s = _Sys()
    s.nrows = K.shape[0]
    s.nnz = len(col)
    s.rowptr = rowptr.ctypes.data_as(C.POINTER(C.c_int64))
    s.col = _ip(col)
    s.K, s.M = _dp(Kv), _dp(Mv)
    return s, (rowptr, col, Kv, Mv)


def apply(system: System, rho: float, x: np.ndarray) -> np.ndarray:
    """y = (rho K + M) x, row by row in column order."""
    s, keep = _sys_struct(system)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    _load().ora_apply(C.byref(s), rho, _dp(x), _dp(y))
    return y


def jacobi_pcg(system: System, rho: float, b: np.ndarray, tol: float = 1e-13,
               maxit: int = 100000, x0: np.ndarray | None = None):
    """Diagonally preconditioned CG in FP64; returns (x, iterations, ||b-Ax||/||b||)."""
    s, keep = _sys_struct(system)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    rr = C.c_double(0.0)
    it = _load().ora_jacobi_pcg(C.byref(s), rho, _dp(b), _dp(x), tol, maxit, C.byref(rr))
    if it < 0:
        raise FloatingPointError("oracle PCG breakdown after %d iterations" % (-it - 1))
    return x, it, rr.value


def cholesky_solve(A_dense: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Own dense Cholesky factorisation and triangular solves."""
    L = np.ascontiguousarray(A_dense, dtype=np.float64).copy()
    n = L.shape[0]
    rc = _load().ora_cholesky(n, _dp(L))
    if rc != 0:
        raise np.linalg.LinAlgError("non-positive pivot %d" % rc)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty(n)
    _load().ora_cholesky_solve(n, _dp(L), _dp(b), _dp(x))
    return x


def errors(system: System, u: np.ndarray, exact: dict, qlevel: int = 1):
    """(||exact - u_h||_L2^2, ||grad(exact - u_h)||_L2^2) by quadrature."""
    U = system.full_vector(u)
    t, keep = _target_struct(exact)
    l2 = C.c_double(0.0); h1 = C.c_double(0.0)
    tets = np.ascontiguousarray(system.tets, dtype=np.int32)
    _load().ora_errors(len(U), _dp(system.xyz), len(tets), _ip(tets), _dp(U), C.byref(t),
                       qlevel, C.byref(l2), C.byref(h1))
    return l2.value, h1.value


def error_hm1(system: System, u: np.ndarray, scale: float = 1.0) -> float:
    """Discrete H^-1 error of w - u_h, w = scale * ubar, ubar the target the system was
    assembled with (the H^-1 column of Tables 3, 6 and 8; the paper does not state its
    discrete form, this is the dual norm on the P1 space with zero boundary values):

        ||w - u_h||_{-1,h}^2 = sup_v (w - u_h, v)^2 / ||grad v||^2 = r^T K^-1 r,
        r_i = (w - u_h, phi_i)_L2 = scale * f_i - (M u)_i,

    with f the system's load vector (its quadrature for the w part) and M, K its mass and
    stiffness matrices; K^-1 r by a sparse direct solve."""
    r = scale * system.f - system.M @ u
    if not np.any(r):
        return 0.0
    y = spla.spsolve(system.K.tocsc(), r)
    return float(r @ y)


def target_values(target: dict, pts: np.ndarray) -> np.ndarray:
    """ubar at the given points (npts x 3)."""
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    t, keep = _target_struct(target)
    out = np.empty(len(pts))
    _load().ora_target_values(C.byref(t), len(pts), _dp(pts), _dp(out))
    return out


def recover(system: System, rho: float, u: np.ndarray, target: dict):
    """Control and adjoint from the state (Sec. 2: the gradient equation gives
    z = (ubar - u) / rho, the adjoint p = -rho u), as nodal values at the unknowns'
    vertices: z_i = (ubar(x_i) - u_i) / rho, p_i = -rho u_i."""
    verts = np.flatnonzero(system.dof >= 0)
    order = np.argsort(system.dof[verts])
    x = system.xyz[verts[order]]
    ub = target_values(target, x)
    z = (ub - u) / rho
    p = -rho * u
    return z, p


def tet_gradients(xyz: np.ndarray, tets: np.ndarray):
    """(volume [nt], barycentric gradients [nt, 4, 3]) of every tet: with E the 3x3 matrix of
    edge vectors x_a - x_0 (rows, a = 1..3), grad lambda_a are the columns of E^{-1} and
    grad lambda_0 = -sum of the others."""
    X = xyz[tets]
    E = X[:, 1:, :] - X[:, :1, :]
    det = np.linalg.det(E)
    G = np.linalg.inv(E).transpose(0, 2, 1)          # row a-1 = grad lambda_a
    g = np.concatenate([-G.sum(axis=1, keepdims=True), G], axis=1)
    return np.abs(det) / 6.0, g


def error_indicator(system: System, rho: float, u: np.ndarray, target: dict, qlevel: int = 1):
    """Residual error indicator of the reaction-diffusion problem -rho Lap u + u = ubar
    (the paper's adaptive runs, Sec. 4.2-4.3, use a residual indicator after Verfurth; this is
    Verfurth's robust estimator for -eps Lap u + u = f with eps = rho), per tet:

        eta_T^2 = a_T^2 ||ubar - u_h||^2_T + 1/2 sum_{interior faces F of T}
                  rho^{-1/2} a_F |F| (rho [grad u_h . n_F])^2,   a_S = min(h_S / sqrt(rho), 1),

    h_T, h_F the longest edge of T and F (Lap u_h = 0 on P1 elements; the jump of the
    normal derivative is constant on a face).  The volume integral uses the rule of
    :func:`qrule` of the given level.  Returns eta_T^2 [nt]."""
    xyz, tets = system.xyz, np.asarray(system.tets, dtype=np.int64)
    U = system.full_vector(u)
    vol, g = tet_gradients(xyz, tets)
    gu = np.einsum("ta,tad->td", U[tets], g)            # grad u_h per tet
    X = xyz[tets]
    edges = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    hT = np.max([np.linalg.norm(X[:, a] - X[:, b], axis=1) for a, b in edges], axis=0)
    aT = np.minimum(hT / np.sqrt(rho), 1.0)
    bary, wt = qrule(qlevel)
    pts = np.einsum("qa,tad->tqd", bary, X)
    ub = target_values(target, pts.reshape(-1, 3)).reshape(len(tets), -1)
    uh = np.einsum("qa,ta->tq", bary, U[tets])
    eta2 = aT ** 2 * vol * ((ub - uh) ** 2 @ wt)
    # interior faces: the face opposite vertex a of each tet, matched by its vertex set
    faces = np.stack([np.delete(tets, a, axis=1) for a in range(4)], axis=1)   # [nt, 4, 3]
    keys = np.sort(faces, axis=2).reshape(-1, 3)
    owner = np.repeat(np.arange(len(tets)), 4)
    order = np.lexsort((keys[:, 2], keys[:, 1], keys[:, 0]))
    k, o = keys[order], owner[order]
    same = np.all(k[1:] == k[:-1], axis=1)
    i1 = np.flatnonzero(same)
    t1, t2 = o[i1], o[i1 + 1]
    F = xyz[k[i1]]                                      # [nf, 3, 3]
    cr = np.cross(F[:, 1] - F[:, 0], F[:, 2] - F[:, 0])
    area = 0.5 * np.linalg.norm(cr, axis=1)
    n = cr / np.linalg.norm(cr, axis=1, keepdims=True)
    jump = np.einsum("fd,fd->f", gu[t1] - gu[t2], n)
    hF = np.max([np.linalg.norm(F[:, a] - F[:, b], axis=1) for a, b in ((0, 1), (0, 2), (1, 2))],
                axis=0)
    aF = np.minimum(hF / np.sqrt(rho), 1.0)
    c = rho ** -0.5 * aF * area * (rho * jump) ** 2
    np.add.at(eta2, t1, 0.5 * c)
    np.add.at(eta2, t2, 0.5 * c)
    return eta2


def dorfler_mark(eta2: np.ndarray, theta: float = 0.5) -> np.ndarray:
    """Bulk marking: the tets with eta_T^2 >= t for the largest t such that the marked tets
    carry at least theta * sum eta^2 (ties at t are all marked; none when every eta is 0)."""
    order = np.sort(eta2)[::-1]
    csum = np.cumsum(order)
    if not csum[-1] > 0.0:
        return np.zeros(len(eta2), dtype=bool)          # nothing to refine
    k = int(np.searchsorted(csum, theta * csum[-1]))
    t = order[min(k, len(order) - 1)]
    return eta2 >= t


def kuhn_rows(n: int, target: dict, rows, xyz: np.ndarray | None = None, qlevel: int = 0):
    """Rows (unknown indices) of K, M and f for selected unknowns, without assembling the mesh.

    Returns (cols [len, 15] with -1 padding, K [len, 15], M [len, 15], f [len])."""
    m = n - 1
    rows = np.asarray(rows, dtype=np.int64)
    i = rows % m + 1
    j = (rows // m) % m + 1
    k = rows // (m * m) + 1
    vtx = np.ascontiguousarray(i + (n + 1) * (j + (n + 1) * k), dtype=np.int64)
    cols = np.empty((len(rows), 15), dtype=np.int32)
    K = np.empty((len(rows), 15))
    M = np.empty((len(rows), 15))
    f = np.empty(len(rows))
    t, keep = _target_struct(target)
    xp = None
    if xyz is not None:
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        xp = _dp(xyz)
    rc = _load().ora_kuhn_rows(n, xp, C.byref(t), qlevel, len(rows),
                               vtx.ctypes.data_as(C.POINTER(C.c_int64)), _ip(cols), _dp(K),
                               _dp(M), _dp(f))
    if rc != 0:
        raise ValueError("kuhn_rows: a vertex is not interior")
    return cols, K, M, f
