"""Rank-based (nonparanormal) sufficient statistics, FP64.

Test infrastructure only (see ``oracle/__init__``).

Paper: Section "The model" adopts the Gaussian-copula (nonparanormality)
assumption and computes {S_l} with the Nonparanormal Skeptic; Section
"Algorithm" describes the COCA form used at scale: replace mat_l[D] by
the matrix of ranks of each of its rows, map the ranks to a normal
distribution and take the singular vectors (the Gram) of that matrix.
The worked example of the appendix "Preserving input sparsity" fixes the
conventions the text leaves open: ties take the lowest rank of their
group (two zeros that would be ranked 2 and 3 both get 2), and rank k of
a row of n entries maps to Phi^-1(k / (n + 1)).

Reading (the paper is silent): the scores are not re-centred or
re-scaled before the Gram, S_l = Z_l Z_l^T with Z_l the score matrix, as
in the worked example.
"""

import numpy as np
from scipy.special import ndtri
from scipy.stats import rankdata

from .gram import matricize


def min_ranks(m: np.ndarray) -> np.ndarray:
    """Rank of every entry within its row (1 = smallest), ties taking the
    lowest rank of their group (the worked example's convention)."""
    return rankdata(np.asarray(m, dtype=np.float64), method="min", axis=1).astype(np.int64)


def normal_scores(m: np.ndarray) -> np.ndarray:
    """Z_ij = Phi^-1(rank_ij / (n + 1)), n = entries per row."""
    m = np.asarray(m, dtype=np.float64)
    n = m.shape[1]
    return ndtri(min_ranks(m) / (n + 1.0))


def zero_scores(m: np.ndarray) -> np.ndarray:
    """z_i: the score every zero of row i maps to (the rank-one term of the
    appendix's sparsity-preserving decomposition Z = (Z - z 1^T) + z 1^T);
    0 for rows without a zero."""
    m = np.asarray(m, dtype=np.float64)
    n = m.shape[1]
    below = (m < 0).sum(axis=1)          # entries ranked ahead of the zeros
    has_zero = (m == 0).any(axis=1)
    return np.where(has_zero, ndtri((below + 1.0) / (n + 1.0)), 0.0)


def skeptic_gram(t: np.ndarray, axis: int) -> np.ndarray:
    """S_l = Z_l Z_l^T, Z_l the normal scores of the rows of mat_l[T]."""
    z = normal_scores(matricize(t, axis))
    return z @ z.T
