"""Oracle restatement of the AMG-preconditioned CG solve (numpy/scipy, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper preconditions CG by one AMG V-cycle with one pre- and one
post-smoothing step (Sec. 3.1, eq. (amgpre); Sec. 4 set-up) and builds the
coarse operators by Galerkin's method A_c = P^T A P (Sec. 3.1).  Its coarsening
(red-black colouring with averaging interpolation) is replaced here by smoothed
aggregation; every rule below is stated in the docstring that applies it, and
the CUDA library follows the same rules in code of its own:

* strength: i != j is a strong pair iff |a_ij| >= theta sqrt(a_ii) sqrt(a_jj) and a_ij != 0;
  a node without strong neighbours is *isolated* and is not aggregated;
* distance-2 maximal independent set by priorities (see :func:`mis2`);
* aggregates: each MIS-2 root with its strong neighbours, then every other node
  joins the phase-1 aggregate it has most strong edges to (ties: smaller id);
* tentative P_t(i, agg(i)) = 1; filtered A_F keeps the diagonal and strong entries;
* P = P_t - omega D^{-1} A_F P_t, omega = 4 / (3 lambda_F), lambda_F the Gershgorin
  bound max_i sum_j |A_F(i,j)| / a_ii;
* coarsest level: dense inverse (from a Cholesky factorisation) in FP64 when it has at
  most coarse_max unknowns; when coarsening stops above that size (every node isolated,
  or too few aggregates) the coarsest level is solved by the smoother alone;
* smoother: Chebyshev of degree k on D^{-1}A over [lambda/ratio, lambda] with lambda the
  Gershgorin bound of D^{-1}A, or one l1-Jacobi step.

The paper's own coarsening is restated as well (``coarsening="kf"``, Sec. 3.1 after
KF1998): red-black colouring (visit the unknowns in a fixed order; an unmarked one
becomes coarse and its unmarked matrix-graph neighbours fine), interpolation of a fine
unknown by the average over its coarse neighbours, Galerkin A_c = P^T A P, and symmetric
Gauss-Seidel smoothing (``smoother="sgs"``: one forward sweep before the coarse-grid
correction, one backward sweep after it).  The paper leaves the visiting order open; here
it is decreasing hash priority (:func:`priority`).  Gauss-Seidel runs in the order of a
greedy colouring of the matrix graph (colour classes in increasing order forward,
decreasing backward; the unknowns of one class do not couple, so their order within the
class does not matter).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

UNDECIDED, IN, OUT = 1, 2, 0
DEFAULTS = dict(theta=0.05, smoother="chebyshev", degree=2, cheb_ratio=6.0,
                coarse_max=256, max_levels=16, seed=0, min_ratio=0.9, coarsening="sa",
                max_row=8192, order="hash")


# ------------------------------------------------------------- utilities

def fmix32(u: np.ndarray) -> np.ndarray:
    """MurmurHash3's 32-bit finaliser (A. Appleby), in wrapping uint32 arithmetic."""
    h = np.asarray(u, dtype=np.uint32).copy()
    with np.errstate(over="ignore"):
        h ^= h >> np.uint32(16)
        h *= np.uint32(0x85EBCA6B)
        h ^= h >> np.uint32(13)
        h *= np.uint32(0xC2B2AE35)
        h ^= h >> np.uint32(16)
    return h


def priority(n: int, seed: int) -> np.ndarray:
    """Priority of node i: (fmix32(i xor s) >> 1) * 2^31 + i, s = 0x9E3779B9 (seed+1) mod 2^32.

    Unique per node, so every comparison below is a strict order."""
    s = np.uint32((0x9E3779B9 * (seed + 1)) & 0xFFFFFFFF)
    i = np.arange(n, dtype=np.uint32)
    h = fmix32(i ^ s).astype(np.uint64)
    return ((h >> np.uint64(1)) << np.uint64(31)) | np.arange(n, dtype=np.uint64)


def rows_of(A) -> np.ndarray:
    return np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))


def spgemm(A, B):
    """C = A B keeping every structural entry (no value-based dropping).

    Products a_ik b_kj are expanded in row order of A, then k order, then the
    order of B's row; they are stably sorted by (i, j) and each run is summed
    left to right."""
    A = sp.csr_matrix(A)
    B = sp.csr_matrix(B)
    nA = np.diff(A.indptr)
    ar = rows_of(A)
    cnt = np.diff(B.indptr)[A.indices]
    tot = int(cnt.sum())
    if tot == 0:
        return sp.csr_matrix((A.shape[0], B.shape[1]))
    pi = np.repeat(ar, cnt)
    av = np.repeat(A.data, cnt)
    start = np.repeat(B.indptr[A.indices], cnt)
    off = np.arange(tot) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    bj = B.indices[start + off]
    bv = B.data[start + off]
    prod = av * bv
    order = np.lexsort((bj, pi))  # stable: keeps expansion order inside (i, j) runs
    pi, bj, prod = pi[order], bj[order], prod[order]
    new = np.ones(tot, dtype=bool)
    new[1:] = (pi[1:] != pi[:-1]) | (bj[1:] != bj[:-1])
    starts = np.flatnonzero(new)
    vals = np.add.reduceat(prod, starts)
    rows = pi[starts]
    cols = bj[starts]
    indptr = np.zeros(A.shape[0] + 1, dtype=np.int64)
    np.add.at(indptr, rows + 1, 1)
    indptr = np.cumsum(indptr)
    del nA
    C = sp.csr_matrix((vals, cols.astype(np.int32), indptr), shape=(A.shape[0], B.shape[1]))
    C.has_sorted_indices = True
    return C


def add_struct(A, B, alpha=1.0, beta=1.0):
    """alpha A + beta B on the union pattern, keeping structural zeros."""
    A = sp.csr_matrix(A).tocoo()
    B = sp.csr_matrix(B).tocoo()
    r = np.concatenate([A.row, B.row])
    c = np.concatenate([A.col, B.col])
    v = np.concatenate([alpha * A.data, beta * B.data])
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    new = np.ones(len(r), dtype=bool)
    new[1:] = (r[1:] != r[:-1]) | (c[1:] != c[:-1])
    st = np.flatnonzero(new)
    vals = np.add.reduceat(v, st) if len(st) else v
    indptr = np.zeros(A.shape[0] + 1, dtype=np.int64)
    np.add.at(indptr, r[st] + 1, 1)
    C = sp.csr_matrix((vals, c[st].astype(np.int32), np.cumsum(indptr)), shape=A.shape)
    C.has_sorted_indices = True
    return C


def diagonal(A) -> np.ndarray:
    A = sp.csr_matrix(A)
    d = np.zeros(A.shape[0])
    r = rows_of(A)
    m = A.indices == r
    d[r[m]] = A.data[m]
    return d


# ------------------------------------------------------------- setup

def strength(A, theta: float) -> np.ndarray:
    """Boolean over A's stored entries: True where (i, j), i != j, is a strong pair:
    |a_ij| >= (theta sqrt(a_ii)) sqrt(a_jj)."""
    d = diagonal(A)
    sq = np.sqrt(d)
    r = rows_of(A)
    c = A.indices
    return (r != c) & (A.data != 0.0) & (np.abs(A.data) >= (theta * sq[r]) * sq[c])


def _segmax(vals, indptr):
    """Per-row maximum of vals over CSR rows (rows with no entries -> 0)."""
    out = np.zeros(len(indptr) - 1, dtype=vals.dtype)
    ne = np.flatnonzero(np.diff(indptr) > 0)
    if len(ne):
        out[ne] = np.maximum.reduceat(vals, indptr[:-1][ne])
    return out


def mis2(S, prio: np.ndarray, isolated: np.ndarray, max_rounds: int = 10000):
    """Distance-2 maximal independent set of the strong graph S (CSR pattern).

    Node i carries the key (state, priority) with IN > UNDECIDED > OUT.  In each
    round every node takes the largest key within graph distance 2 (two passes of
    "max over self and neighbours"); an UNDECIDED node whose own key is that
    maximum enters the set, and an UNDECIDED node whose maximum belongs to a node
    already in the set leaves.  Isolated nodes start as OUT.  The result equals
    the greedy set that scans nodes by decreasing priority."""
    n = S.shape[0]
    state = np.where(isolated, OUT, UNDECIDED).astype(np.uint64)
    for _ in range(max_rounds):
        und = state == UNDECIDED
        if not und.any():
            return state
        key = (state << np.uint64(62)) | prio
        m1 = np.maximum(key, _segmax(key[S.indices], S.indptr))
        m2 = np.maximum(m1, _segmax(m1[S.indices], S.indptr))
        new_in = und & (m2 == key)
        new_out = und & ~new_in & ((m2 >> np.uint64(62)) == IN)
        state[new_in] = IN
        state[new_out] = OUT
    raise RuntimeError("MIS-2 did not finish")


def aggregate(A, theta: float, seed: int):
    """(agg, nagg, strong_mask): agg[i] = aggregate of node i, -1 for isolated nodes."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    smask = strength(A, theta)
    r = rows_of(A)
    deg = np.bincount(r[smask], minlength=n)
    isolated = deg == 0
    S = sp.csr_matrix((np.ones(int(smask.sum())), A.indices[smask], np.concatenate(
        [[0], np.cumsum(deg)])), shape=(n, n))
    state = mis2(S, priority(n, seed), isolated)
    roots = state == IN
    aggid = np.cumsum(roots) - 1
    nagg = int(roots.sum())
    agg = np.full(n, -1, dtype=np.int64)
    agg[roots] = aggid[roots]
    # phase 1: strong neighbours of a root join it (unique: roots are >= 3 apart)
    sr = rows_of(S)
    sc = S.indices
    e1 = roots[sc] & ~roots[sr]
    if e1.any():
        assert len(np.unique(sr[e1])) == int(e1.sum()), "node adjacent to two MIS-2 roots"
        agg[sr[e1]] = aggid[sc[e1]]
    phase1 = agg >= 0
    # phase 2: the rest joins the phase-1 aggregate with most strong edges to it
    e2 = (~phase1[sr]) & (~isolated[sr]) & phase1[sc]
    if e2.any():
        ri, ai = sr[e2], agg[sc[e2]]
        order = np.lexsort((ai, ri))
        ri, ai = ri[order], ai[order]
        new = np.ones(len(ri), dtype=bool)
        new[1:] = (ri[1:] != ri[:-1]) | (ai[1:] != ai[:-1])
        st = np.flatnonzero(new)
        counts = np.diff(np.append(st, len(ri)))
        ur, ua = ri[st], ai[st]
        best = np.lexsort((ua, -counts, ur))
        ur, ua = ur[best], ua[best]
        first = np.ones(len(ur), dtype=bool)
        first[1:] = ur[1:] != ur[:-1]
        agg[ur[first]] = ua[first]
    if ((agg < 0) & ~isolated).any():
        raise RuntimeError("aggregation left a non-isolated node unassigned")
    return agg, nagg, smask


def tentative(agg: np.ndarray, nagg: int):
    n = len(agg)
    m = agg >= 0
    indptr = np.concatenate([[0], np.cumsum(m)])
    P = sp.csr_matrix((np.ones(int(m.sum())), agg[m].astype(np.int32), indptr), shape=(n, nagg))
    P.has_sorted_indices = True
    return P


def filtered(A, smask):
    """A_F: the diagonal and the strong entries of A (weak entries dropped, not lumped)."""
    A = sp.csr_matrix(A)
    r = rows_of(A)
    keep = smask | (A.indices == r)
    cnt = np.bincount(r[keep], minlength=A.shape[0])
    F = sp.csr_matrix((A.data[keep], A.indices[keep], np.concatenate([[0], np.cumsum(cnt)])),
                      shape=A.shape)
    F.has_sorted_indices = True
    return F


def gershgorin(A) -> float:
    """max_i sum_j |a_ij| / a_ii, an upper bound of the spectrum of D^{-1} A."""
    A = sp.csr_matrix(A)
    d = diagonal(A)
    s = np.add.reduceat(np.abs(A.data), A.indptr[:-1]) if A.nnz else np.zeros(A.shape[0])
    s[np.diff(A.indptr) == 0] = 0.0
    return float(np.max(s / d)) if A.shape[0] else 0.0


def smoothed_prolongator(A, smask, agg, nagg):
    Pt = tentative(agg, nagg)
    F = filtered(A, smask)
    lam = gershgorin(F)
    omega = 4.0 / (3.0 * lam)
    dinv = 1.0 / diagonal(A)
    DF = sp.csr_matrix((F.data * np.repeat(dinv, np.diff(F.indptr)), F.indices, F.indptr),
                       shape=F.shape)
    B = spgemm(DF, Pt)
    return add_struct(Pt, B, 1.0, -omega), omega


# ------------------------------------------------------------- red-black coarsening

def neighbours(A, i):
    """Matrix-graph neighbours of i: columns j != i of stored nonzero a_ij (column order)."""
    lo, hi = A.indptr[i], A.indptr[i + 1]
    cols = A.indices[lo:hi]
    vals = A.data[lo:hi]
    return cols[(cols != i) & (vals != 0.0)]


def red_black(A, seed: int, order: str = "hash") -> np.ndarray:
    """Red-black colouring (Sec. 3.1, after KF1998 Algorithm 2): visit the unknowns by
    decreasing priority (order "hash"), or by increasing index (order "natural"); an
    unmarked one is marked black (coarse) and its unmarked neighbours red (fine).  Returns
    the boolean coarse mask."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    mark = np.zeros(n, dtype=np.int8)  # 0 unmarked, 1 black, 2 red
    visit = np.arange(n) if order == "natural" else np.argsort(priority(n, seed))[::-1]
    for i in visit:  # priorities are unique
        if mark[i]:
            continue
        mark[i] = 1
        nb = neighbours(A, i)
        mark[nb[mark[nb] == 0]] = 2
    return mark == 1


def averaging_prolongator(A, coarse: np.ndarray):
    """P: a coarse unknown keeps its value (P(i, c(i)) = 1, coarse unknowns numbered in
    increasing order); a fine unknown is the average over its coarse neighbours
    (P(i, c(j)) = 1 / #C_i for j in C_i) (Sec. 3.1)."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    cid = np.cumsum(coarse) - 1
    rows, cols, vals = [], [], []
    for i in range(n):
        if coarse[i]:
            rows.append(i)
            cols.append(cid[i])
            vals.append(1.0)
            continue
        nb = neighbours(A, i)
        cn = nb[coarse[nb]]
        if len(cn) == 0:
            raise RuntimeError("fine unknown without a coarse neighbour")
        w = 1.0 / len(cn)
        for j in cn:
            rows.append(i)
            cols.append(cid[j])
            vals.append(w)
    P = sp.csr_matrix((np.array(vals), (np.array(rows), np.array(cols))),
                      shape=(n, int(coarse.sum())))
    P.sort_indices()
    return P


def greedy_colouring(A, seed: int) -> np.ndarray:
    """Colour of each unknown: visit by decreasing priority and take the smallest colour
    not used by an already coloured neighbour."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    col = np.full(n, -1, dtype=np.int64)
    for i in np.argsort(priority(n, seed))[::-1]:  # priorities are unique
        used = set(col[neighbours(A, i)].tolist())
        c = 0
        while c in used:
            c += 1
        col[i] = c
    return col


def gauss_seidel(A, b, x, colours, forward: bool):
    """One Gauss-Seidel sweep in colour order: for each colour class (increasing when
    forward, decreasing otherwise) x_i = (b_i - sum_{j != i} a_ij x_j) / a_ii, the sum over
    A's stored entries in column order."""
    A = sp.csr_matrix(A)
    d = diagonal(A)
    off = A.copy()
    off.setdiag(0.0)
    off.eliminate_zeros()
    x = np.zeros_like(b) if x is None else x.copy()
    ncol = int(colours.max()) + 1 if len(colours) else 0
    order = range(ncol) if forward else range(ncol - 1, -1, -1)
    for c in order:
        idx = np.flatnonzero(colours == c)
        x[idx] = (b[idx] - off[idx] @ x) / d[idx]
    return x


class Level:
    pass


def _longest_row(B) -> int:
    """Most stored entries in a row of a CSR matrix (0 for no rows)."""
    return int(np.diff(B.indptr).max()) if B.shape[0] else 0


def build_hierarchy(A, opts: dict | None = None, K=None, M=None):
    """Smoothed-aggregation hierarchy of A.  With K and M given (A = rho K + M),
    the coarse pencils K_l = P^T K P and M_l = P^T M P are kept as well."""
    o = dict(DEFAULTS)
    if opts:
        o.update(opts)
    levels = []
    Al = sp.csr_matrix(A)
    Kl, Ml = K, M
    for lev in range(o["max_levels"]):
        L = Level()
        L.A = Al
        L.K, L.M = Kl, Ml
        L.dinv = 1.0 / diagonal(Al)
        L.lmax = gershgorin(Al)
        L.l1 = np.add.reduceat(np.abs(Al.data), Al.indptr[:-1])
        levels.append(L)
        n = Al.shape[0]
        if o["smoother"] == "sgs":
            L.colours = greedy_colouring(Al, o["seed"] + lev)
        last = n <= o["coarse_max"] or lev == o["max_levels"] - 1
        kf = o["coarsening"] == "kf"
        if not last:
            if kf:
                coarse = red_black(Al, o["seed"] + lev, o["order"])
                nagg = int(coarse.sum())
            else:
                agg, nagg, smask = aggregate(Al, o["theta"], o["seed"] + lev)
            if nagg == 0 or nagg >= o["min_ratio"] * n:
                last = True
        if last:
            L.coarsest = True
            if n <= o["coarse_max"]:
                Lc = np.linalg.cholesky(Al.toarray())
                Li = np.linalg.inv(Lc)
                L.Ainv = Li.T @ Li
            else:
                L.Ainv = None  # smoother-only coarsest level
            return levels
        L.coarsest = False
        if kf:
            L.coarse, L.nagg = coarse, nagg
            L.P = averaging_prolongator(Al, coarse)
        else:
            L.agg, L.nagg = agg, nagg
            L.P, L.omega = smoothed_prolongator(Al, smask, agg, nagg)
        L.R = sp.csr_matrix(L.P.T)
        L.R.sort_indices()
        AP = spgemm(Al, L.P)
        Ac = spgemm(L.R, AP)
        if max(_longest_row(L.R), _longest_row(AP), _longest_row(Ac)) > o["max_row"]:
            # the restriction or a Galerkin product would have a row longer than max_row
            # (dense coarse levels): this level is the coarsest instead
            L.coarsest = True
            L.P = L.R = None
            if n <= o["coarse_max"]:
                Lc = np.linalg.cholesky(Al.toarray())
                Li = np.linalg.inv(Lc)
                L.Ainv = Li.T @ Li
            else:
                L.Ainv = None
            return levels
        Al = Ac
        if K is not None:
            Kl = spgemm(L.R, spgemm(Kl, L.P))
            Ml = spgemm(L.R, spgemm(Ml, L.P))
    return levels


# ------------------------------------------------------------- smoothing

def chebyshev(A, dinv, b, x, lmax, ratio, degree):
    """Degree-k Chebyshev iteration on D^{-1} A x = D^{-1} b over [lmax/ratio, lmax]
    (three-term recurrence of Y. Saad, Iterative Methods, Alg. 12.1).  x=None means
    the zero initial guess."""
    a, bb = lmax / ratio, lmax
    theta, delta = 0.5 * (bb + a), 0.5 * (bb - a)
    sigma = theta / delta
    if x is None:
        x = np.zeros_like(b)
        r = dinv * b
    else:
        x = x.copy()
        r = dinv * (b - A @ x)
    rho_old = 1.0 / sigma
    d = r / theta
    for step in range(1, degree + 1):
        x = x + d
        if step == degree:
            break
        r = r - dinv * (A @ d)
        rho_new = 1.0 / (2.0 * sigma - rho_old)
        d = (rho_new * rho_old) * d + (2.0 * rho_new / delta) * r
        rho_old = rho_new
    return x


def l1_jacobi(A, l1, b, x):
    if x is None:
        return b / l1
    return x + (b - A @ x) / l1


def smooth(L, b, x, o, forward=True):
    if o["smoother"] == "chebyshev":
        return chebyshev(L.A, L.dinv, b, x, L.lmax, o["cheb_ratio"], o["degree"])
    if o["smoother"] == "sgs":
        return gauss_seidel(L.A, b, x, L.colours, forward)
    return l1_jacobi(L.A, L.l1, b, x)


def vcycle(levels, b, opts: dict | None = None, lev: int = 0):
    """One V-cycle with zero initial guess: pre-smooth, residual, restrict,
    recurse, prolong, post-smooth (Sec. 3.1, eq. (amgpre), applied recursively)."""
    o = dict(DEFAULTS)
    if opts:
        o.update(opts)
    L = levels[lev]
    if L.coarsest:
        if L.Ainv is not None:
            return L.Ainv @ b
        x = smooth(L, b, None, o, forward=True)
        if o["smoother"] == "sgs":  # both sweeps meet here: keep the V-cycle symmetric
            x = smooth(L, b, x, o, forward=False)
        return x
    x = smooth(L, b, None, o, forward=True)
    r = b - L.A @ x
    xc = vcycle(levels, L.R @ r, o, lev + 1)
    x = x + L.P @ xc
    return smooth(L, b, x, o, forward=False)


# ------------------------------------------------------------- Krylov

def pcg(A, b, prec=None, tol=1e-8, maxit=1000, flexible=False, x0=None):
    """Preconditioned CG (Hestenes-Stiefel).  With flexible=True, beta is the
    Polak-Ribiere form <z_{k+1}, r_{k+1} - r_k> / <z_k, r_k> (flexible CG).
    Stops when ||r||_2 <= tol ||b||_2.  Returns (x, iterations, true relres, history)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A @ x
    bn = np.linalg.norm(b) or 1.0
    z = prec(r) if prec else r.copy()
    p = z.copy()
    rz = r @ z
    hist = [np.linalg.norm(r) / bn]
    it = 0
    while it < maxit and hist[-1] > tol:
        q = A @ p
        pq = p @ q
        if not pq > 0:
            raise FloatingPointError("PCG breakdown: <p, Ap> = %r" % pq)
        alpha = rz / pq
        x = x + alpha * p
        r_old = r
        r = r - alpha * q
        z = prec(r) if prec else r.copy()
        rz_new = r @ z
        beta = ((rz_new - r_old @ z) / rz) if flexible else (rz_new / rz)
        rz = rz_new
        p = z + beta * p
        it += 1
        hist.append(np.linalg.norm(r) / bn)
    relres = np.linalg.norm(b - A @ x) / bn
    return x, it, relres, hist
