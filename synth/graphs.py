"""Planted sparse precision matrices (ground-truth graphs for synthetic data)."""

import numpy as np


def er_precision(d: int, deg: float, rng: np.random.Generator,
                 wlo: float = 0.1, whi: float = 0.5) -> np.ndarray:
    """Erdos-Renyi precision matrix of size d x d (float64).

    Edges appear independently with probability deg/(d-1); each edge weight is
    U[wlo, whi] with a random sign; the diagonal is |row sum| + 1, which makes
    the matrix strictly diagonally dominant and hence positive definite.
    """
    if d < 2:
        return np.ones((d, d))
    p = min(1.0, deg / (d - 1))
    mask = np.triu(rng.random((d, d)) < p, k=1)
    w = rng.uniform(wlo, whi, size=(d, d)) * np.where(rng.random((d, d)) < 0.5, -1.0, 1.0)
    up = np.where(mask, w, 0.0)
    psi = up + up.T
    np.fill_diagonal(psi, np.abs(psi).sum(axis=1) + 1.0)
    return psi
