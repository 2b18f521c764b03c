"""End-to-end FP64 fit for a two-axis matrix (Algorithm 1, in order).

Test infrastructure only (see ``oracle/__init__``).
"""

from dataclasses import dataclass

import numpy as np

from .gram import gram
from .recon import topk_rows
from .solve import KSProblem, solve_newton, two_axis_problem
from .spectra import dual_lift, top_eigh, two_axis_spectra


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


@dataclass
class MultiAxisFit:
    E: list        # per axis, descending
    V: list        # per axis, eigenvectors as columns
    lam: list      # per axis
    info: object
    topk: list     # per axis (idx, val)


def fit_multimodal(xs, r_cells, ks, eps=None, tol=1e-12, sample_rows=None):
    """Several modalities X_m (cells x p_m, centred) sharing the cell axis.

    Section "Algorithm": the Gram of an axis shared by several modalities is
    the sum of their Grams, i.e. the Gram of the concatenation [X_1 X_2 ...];
    its top eigenpairs come from the concatenation's column Gram through the
    dual lift.  Each modality's own axis takes the full spectrum of
    X_m^T X_m (a diagonal block of that column Gram).  Axes: 0 = cells, m + 1
    = modality m's features; modality m couples axes (0, m + 1).  ks: k per
    axis."""
    xc = np.concatenate([np.asarray(x, dtype=np.float64) for x in xs], axis=1)
    s = xc.T @ xc
    e_c, w_c = top_eigh(s, r_cells)
    E, V = [e_c], [dual_lift(xc, w_c, e_c)]
    off = 0
    for x in xs:
        p = x.shape[1]
        e, w = top_eigh(s[off:off + p, off:off + p], p)
        E.append(e)
        V.append(w)
        off += p
    prob = KSProblem(E, [(0, m + 1) for m in range(len(xs))], eps)
    lam, info = solve_newton(prob, tol=tol)
    lams = prob.split(lam)
    topk = [topk_rows(V[0], lams[0], ks[0], rows=sample_rows)]
    topk += [topk_rows(V[a], lams[a], ks[a]) for a in range(1, len(V))]
    return MultiAxisFit(E, V, lams, info, topk)


def fit_tensor(t, ks, eps=None, tol=1e-12):
    """One K-axis tensor (Notation: S_l = mat_l[T] mat_l[T]^T for every axis),
    full spectrum on every axis, one modality over all axes (the gauge rule
    applies when the traces are equal, as they are at full ranks).  ks: k per
    axis, None for no network on that axis."""
    t = np.asarray(t, dtype=np.float64)
    E, V = [], []
    for a in range(t.ndim):
        e, w = top_eigh(gram(t, a), t.shape[a])
        E.append(e)
        V.append(w)
    prob = KSProblem(E, [tuple(range(t.ndim))], eps)
    lam, info = solve_newton(prob, tol=tol)
    lams = prob.split(lam)
    topk = [topk_rows(V[a], lams[a], ks[a]) if ks[a] else None for a in range(t.ndim)]
    return MultiAxisFit(E, V, lams, info, topk)
