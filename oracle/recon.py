"""Recomposition and per-row top-k thresholding (FP64).

Test infrastructure only (see ``oracle/__init__``).

Algorithm 1, last loop: Psi_l = thresh_{n_l}[V_l Lam_l V_l^T], thresholded
while recomposing so the dense d_l x d_l matrix is never needed at once.
Readings where the paper is silent: the strength of an edge is |Psi_ij|; the
diagonal is never an edge; the threshold keeps the k largest per row (lists
are directed, not symmetrised); equal magnitudes are ordered by the lower
column index.
"""

import numpy as np


def recompose(v: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """Dense Psi = V diag(lam) V^T (only for small d)."""
    v = np.asarray(v, dtype=np.float64)
    return (v * np.asarray(lam, dtype=np.float64)[None, :]) @ v.T


def topk_rows(v: np.ndarray, lam: np.ndarray, k: int, rows=None, block: int = 256):
    """Per-row top-k of |Psi_ij|, j != i, for Psi = V diag(lam) V^T.

    Returns (idx int64 [m, k], val float64 [m, k]) for the requested rows
    (default: all), sorted by |value| descending, ties by lower column index.
    The row block of Psi is formed exactly in FP64 and discarded."""
    v = np.asarray(v, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    d = v.shape[0]
    if not 0 < k < d:
        raise ValueError("need 0 < k < d")
    rows = np.arange(d) if rows is None else np.asarray(rows, dtype=np.int64)
    idx = np.empty((len(rows), k), dtype=np.int64)
    val = np.empty((len(rows), k), dtype=np.float64)
    vl = v * lam[None, :]
    cols = np.arange(d)
    for b0 in range(0, len(rows), block):
        rb = rows[b0:b0 + block]
        psi = vl[rb] @ v.T
        for t, i in enumerate(rb):
            a = np.abs(psi[t])
            a[i] = -np.inf
            order = np.lexsort((cols, -a))[:k]
            idx[b0 + t] = order
            val[b0 + t] = psi[t, order]
    return idx, val


def topk_gap(v: np.ndarray, lam: np.ndarray, k: int, rows=None, block: int = 256):
    """Relative gap (|psi|_k - |psi|_{k+1}) / |psi|_k per requested row, the
    quantity that decides whether the top-k set is numerically determined."""
    v = np.asarray(v, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    d = v.shape[0]
    rows = np.arange(d) if rows is None else np.asarray(rows, dtype=np.int64)
    gap = np.empty(len(rows))
    vl = v * lam[None, :]
    for b0 in range(0, len(rows), block):
        rb = rows[b0:b0 + block]
        psi = np.abs(vl[rb] @ v.T)
        for t, i in enumerate(rb):
            a = psi[t].copy()
            a[i] = -np.inf
            if k + 1 <= d - 1:
                part = -np.partition(-a, k)[:k + 1]
                part = np.sort(part)[::-1]
                gap[b0 + t] = (part[k - 1] - part[k]) / max(part[k - 1], 1e-300)
            else:
                gap[b0 + t] = np.inf
    return gap


def _edge_order(mag: np.ndarray, i: np.ndarray, j: np.ndarray) -> np.ndarray:
    """Indices sorting edges by |value| descending, then (i, j) ascending."""
    return np.lexsort((j, i, -mag))


def topn_edges(v: np.ndarray, lam: np.ndarray, n: int, block: int = 256):
    """The n strongest edges of Psi = V diag(lam) V^T over unordered pairs
    i < j: the global threshold thresh_{n_l} of Algorithm 1's last loop
    (the complexity appendix keeps it with a heap of size n_l).  Returns
    (i, j, value) arrays sorted by |value| descending, ties by (i, j)
    ascending.  Row blocks of Psi are formed exactly in FP64."""
    v = np.asarray(v, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    d = v.shape[0]
    if not 0 < n <= d * (d - 1) // 2:
        raise ValueError("need 0 < n <= d (d - 1) / 2")
    vl = v * lam[None, :]
    bi = np.empty(0, np.int64)
    bj = np.empty(0, np.int64)
    bv = np.empty(0)
    for r0 in range(0, d, block):
        rows = np.arange(r0, min(d, r0 + block))
        psi = vl[rows] @ v.T
        ii, jj = np.nonzero(np.arange(d)[None, :] > rows[:, None])
        ci = rows[ii]
        cv = psi[ii, jj]
        bi, bj, bv = np.concatenate([bi, ci]), np.concatenate([bj, jj]), np.concatenate([bv, cv])
        keep = _edge_order(np.abs(bv), bi, bj)[:n]
        bi, bj, bv = bi[keep], bj[keep], bv[keep]
    return bi, bj, bv


def topn_from_row_lists(idx: np.ndarray, val: np.ndarray, n: int):
    """Global top-n edges from per-row top-k lists (idx, val: d x k, row i
    holding its k strongest off-diagonal entries, as ``topk_rows`` returns
    them): the union of the lists as unordered pairs, its n strongest in the
    order of ``topn_edges``, and whether that is certified to be the global
    top-n.  It is when every row's k-th magnitude lies strictly below the
    n-th magnitude of the union (no row can then hold an edge that strong
    outside its own list), or when every list holds all d - 1 columns.
    Returns (i, j, value, certified)."""
    idx = np.asarray(idx, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    d, k = idx.shape
    rows = np.repeat(np.arange(d), k)
    cols = idx.ravel()
    vals = val.ravel()
    i = np.minimum(rows, cols)
    j = np.maximum(rows, cols)
    _, first = np.unique(i * d + j, return_index=True)  # each pair once
    i, j, vals = i[first], j[first], vals[first]
    order = _edge_order(np.abs(vals), i, j)[:n]
    i, j, vals = i[order], j[order], vals[order]
    if len(vals) < n:
        return i, j, vals, False
    if k == d - 1:
        return i, j, vals, True
    kth = np.abs(val[:, k - 1])
    return i, j, vals, bool(np.all(kth < abs(vals[-1])))
