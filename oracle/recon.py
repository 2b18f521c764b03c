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
