"""Helpers of the GPU tests: move CSR4 exports of the CUDA library into scipy."""
import numpy as np
import scipy.sparse as sp
import torch


def csr4_to_scipy(rowptr, col, val, nrows, ncols):
    """Drop the (col -1, value 0) padding of a CSR4 export."""
    rowptr = rowptr.cpu().numpy().astype(np.int64)
    col = col.cpu().numpy()
    val = val.cpu().numpy()
    rows = np.repeat(np.arange(nrows), np.diff(rowptr))
    keep = col >= 0
    M = sp.csr_matrix((val[keep], (rows[keep], col[keep])), shape=(nrows, ncols))
    M.sort_indices()
    # structure check: real entries sorted and unique inside each row, padding at the end
    return M


def export_system(fa, sys_, which=0):
    info = fa.fem_system_get_info(sys_)
    N, nnz = info["N"], info["nnz"]
    rp = torch.empty(N + 1, dtype=torch.int32, device="cuda")
    ci = torch.empty(nnz, dtype=torch.int32, device="cuda")
    va = torch.empty(nnz, dtype=torch.float64, device="cuda")
    fa.fem_system_export(sys_, which, rp, ci, va)
    return csr4_to_scipy(rp, ci, va, N, N), (rp, ci, va)


def export_level(fa, h, level, which, nrows, ncols):
    nnz = fa.amg_hier_export(h, level, which)
    rp = torch.empty(nrows + 1, dtype=torch.int32, device="cuda")
    ci = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
    va = torch.empty(max(nnz, 1), dtype=torch.float64, device="cuda")
    fa.amg_hier_export(h, level, which, rp, ci, va)
    return csr4_to_scipy(rp, ci[:nnz], va[:nnz], nrows, ncols)


def export_aggregates(fa, h, level, n):
    a = torch.empty(n, dtype=torch.int32, device="cuda")
    fa.amg_hier_export(h, level, 3, None, a, None)
    return a.cpu().numpy().astype(np.int64)


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def sparse_rel(A, B):
    D = (A - B)
    d = np.sqrt((D.multiply(D)).sum()) if D.nnz else 0.0
    nb = np.sqrt((B.multiply(B)).sum())
    return d / nb


def entrywise_rel(A, B):
    """Largest |a_ij - b_ij| over entries of the same pattern, each divided by the largest
    |b_ik| of its row."""
    A = A.tocsr()
    B = B.tocsr()
    D = abs(A - B).tocsr()
    if D.nnz == 0:
        return 0.0
    rmax = abs(B).max(axis=1).toarray().ravel()
    rows = np.repeat(np.arange(D.shape[0]), np.diff(D.indptr))
    return float(np.max(D.data / np.where(rmax[rows] > 0, rmax[rows], 1.0)))
