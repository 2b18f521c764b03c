"""Statistics of a sparse count matrix without densifying it (FP64).

Test infrastructure only (see ``oracle/__init__``).

Paper: the appendix "Preserving input sparsity" writes a transformed
matrix as a matrix with the input's sparsity plus a rank-one term (a
constant per row, z 1^T) and works with the two parts separately.  The
workload's own transform has that form: log1p keeps every zero at zero, and
centring the columns subtracts the rank-one 1 mu^T.  So

    X_c = X - 1 mu^T,  X = log1p(counts) (sparse),  mu = column means,
    X_c^T X_c = X^T X - n mu mu^T          (the column Gram),
    X_c W D = X W D - 1 (mu^T W D)         (the dual lift, D = diag(E)^-1/2),

and neither the Gram nor the lift needs the dense X_c.
"""

import numpy as np
import scipy.sparse as sp


def log1p_sparse(counts) -> sp.csr_matrix:
    """log1p of a sparse count matrix: the same sparsity pattern."""
    c = sp.csr_matrix(counts, dtype=np.float64)
    return sp.csr_matrix((np.log1p(c.data), c.indices, c.indptr), shape=c.shape)


def centred_gram_sparse(x: sp.spmatrix):
    """(X_c^T X_c, mu) for X_c = X - 1 mu^T, mu the column means of X,
    from the sparse X and a rank-one correction."""
    x = sp.csr_matrix(x, dtype=np.float64)
    n = x.shape[0]
    mu = np.asarray(x.sum(axis=0)).ravel() / n
    g = (x.T @ x).toarray()
    return g - n * np.outer(mu, mu), mu


def centred_lift_sparse(x: sp.spmatrix, mu: np.ndarray, w: np.ndarray, e: np.ndarray) -> np.ndarray:
    """X_c W diag(E)^-1/2 from the sparse X and a rank-one correction."""
    x = sp.csr_matrix(x, dtype=np.float64)
    wd = np.asarray(w, dtype=np.float64) / np.sqrt(np.asarray(e, dtype=np.float64))[None, :]
    return x @ wd - np.outer(np.ones(x.shape[0]), mu @ wd)
