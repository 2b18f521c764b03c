"""Kronecker sums and the dense likelihood, for brute-force pins on tiny inputs.

Test infrastructure only (see ``oracle/__init__``).

Introduction: F (+) G := F (x) I + I (x) G, and the model
vec[X] ~ N(0, (Psi_cols (+) Psi_rows)^-1) for X with rows on axis 1 (cells)
and columns on axis 2 (genes).  The appendix "Derivation of the probability
distribution" writes the density with the pseudo-determinant over the span of
the retained eigenvectors, and the exponent as sum_l tr[S_l Psi_l].
"""

import numpy as np


def kron_sum(f: np.ndarray, g: np.ndarray) -> np.ndarray:
    """F (+) G = F (x) I_g + I_f (x) G."""
    return np.kron(f, np.eye(g.shape[0])) + np.kron(np.eye(f.shape[0]), g)


def vec(x: np.ndarray) -> np.ndarray:
    """Column-stacking vectorisation (the convention under which
    vec[A X B^T] = (B (x) A) vec[X])."""
    return np.asarray(x).reshape(-1, order="F")


def dense_nll_full(x: np.ndarray, psi_rows: np.ndarray, psi_cols: np.ndarray) -> float:
    """-2 log-likelihood (constants dropped) of one matrix draw X under the
    full-rank Kronecker-sum model, from explicit d1 d2 x d1 d2 matrices:
    vec[X]^T (Psi_cols (+) Psi_rows) vec[X] - log det(Psi_cols (+) Psi_rows)."""
    omega = kron_sum(psi_cols, psi_rows)
    sign, logdet = np.linalg.slogdet(omega)
    if sign <= 0:
        return np.inf
    v = vec(x)
    return float(v @ omega @ v - logdet)


def dense_nll_singular(x: np.ndarray, v_rows: np.ndarray, lam: np.ndarray,
                       v_cols: np.ndarray, mu: np.ndarray) -> float:
    """-2 log-likelihood of the singular model with Psi_l = V_l diag(.) V_l^T
    (V_l with orthonormal columns, possibly truncated), from explicit matrices:
    the pseudo-log-determinant of the projected Kronecker sum
    P (Psi_cols (+) Psi_rows) P, P = (V_cols V_cols^T) (x) (V_rows V_rows^T),
    taken over its nonzero eigenvalues, and the quadratic form
    tr[S_rows Psi_rows] + tr[S_cols Psi_cols] with S_rows = X X^T,
    S_cols = X^T X."""
    psi_r = (v_rows * lam[None, :]) @ v_rows.T
    psi_c = (v_cols * mu[None, :]) @ v_cols.T
    pr = v_rows @ v_rows.T
    pc = v_cols @ v_cols.T
    proj = np.kron(pc, pr)
    omega = proj @ kron_sum(psi_c, psi_r) @ proj
    ev = np.linalg.eigvalsh(0.5 * (omega + omega.T))
    rank = v_rows.shape[1] * v_cols.shape[1]
    top = np.sort(ev)[::-1][:rank]
    if np.any(top <= 0):
        return np.inf
    quad = np.trace((x @ x.T) @ psi_r) + np.trace((x.T @ x) @ psi_c)
    return float(quad - np.sum(np.log(top)))
