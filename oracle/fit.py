"""End-to-end FP64 fit for a two-axis matrix (Algorithm 1, in order).

Test infrastructure only (see ``oracle/__init__``).
"""

from dataclasses import dataclass

import numpy as np

from .recon import topk_rows
from .solve import solve_newton, two_axis_problem
from .spectra import two_axis_spectra


@dataclass
class TwoAxisFit:
    e_rows: np.ndarray
    v_rows: np.ndarray
    e_cols: np.ndarray
    v_cols: np.ndarray
    lam_rows: np.ndarray
    lam_cols: np.ndarray
    info: object
    topk_rows: tuple
    topk_cols: tuple


def fit_two_axis(x, r_rows, r_cols, k_rows, k_cols, eps=None, tol=1e-12,
                 sample_rows=None):
    """Spectra of both axes, the eigenvalue solve, then per-row top-k of both
    recomposed precisions (rows restricted to ``sample_rows`` if given)."""
    e_r, v_r, e_c, v_c = two_axis_spectra(x, r_rows, r_cols)
    prob = two_axis_problem(e_r, e_c, eps)
    lam, info = solve_newton(prob, tol=tol)
    lr, lc = prob.split(lam)
    tr = topk_rows(v_r, lr, k_rows, rows=sample_rows)
    tc = topk_rows(v_c, lc, k_cols)
    return TwoAxisFit(e_r, v_r, e_c, v_c, lr, lc, info, tr, tc)
