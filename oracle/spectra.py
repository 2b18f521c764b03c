"""Per-axis spectra (FP64).

Test infrastructure only (see ``oracle/__init__``).

Theorem 1: the top-r eigenvectors of S_l are eigenvectors of the MLE Psi_l.
Algorithm 1 takes them as the top-r left singular vectors of D_l, with
E_l = (top-r singular values)^2.  For a two-axis matrix X (cells x genes) the
nonzero spectra of X X^T and X^T X coincide, so E_cells is the top-r of the
gene-Gram spectrum and the cell vectors are lifted through X:
U_r = X W_r diag(sigma_r)^-1, sigma_r^2 = E_r.
"""

import numpy as np


def top_eigh(s: np.ndarray, r: int):
    """Top-r eigenpairs of a symmetric matrix, eigenvalues descending
    (LAPACK syevd through numpy)."""
    w, v = np.linalg.eigh(np.asarray(s, dtype=np.float64))
    order = np.argsort(w)[::-1][:r]
    return w[order], v[:, order]


def dual_lift(x: np.ndarray, w_r: np.ndarray, e_r: np.ndarray) -> np.ndarray:
    """Left singular vectors of X from right ones: X W_r diag(E_r)^-1/2."""
    return (np.asarray(x, dtype=np.float64) @ w_r) / np.sqrt(e_r)[None, :]


def two_axis_spectra(x: np.ndarray, r_rows: int, r_cols: int):
    """Spectra of both axes of a matrix X (rows x cols) through the small
    column Gram: returns (E_rows, V_rows, E_cols, V_cols)."""
    s = np.asarray(x, dtype=np.float64).T @ np.asarray(x, dtype=np.float64)
    e_all, w_all = top_eigh(s, s.shape[0])
    e_cols, v_cols = e_all[:r_cols], w_all[:, :r_cols]
    e_rows = e_all[:r_rows]
    v_rows = dual_lift(x, w_all[:, :r_rows], e_rows)
    return e_rows, v_rows, e_cols, v_cols


def dual_lift_blocks(chunks, mu: np.ndarray, w_r: np.ndarray, e_r: np.ndarray) -> np.ndarray:
    """``dual_lift`` of the centred log1p matrix given as row blocks of
    counts: each block is log1p-transformed, centred by the column means mu
    and multiplied by W_r diag(E_r)^-1/2; the blocks' rows are stacked."""
    wd = np.asarray(w_r, dtype=np.float64) / np.sqrt(np.asarray(e_r, dtype=np.float64))[None, :]
    out = [(np.log1p(np.asarray(c, dtype=np.float64)) - mu[None, :]) @ wd for c in chunks]
    return np.concatenate(out, axis=0)
