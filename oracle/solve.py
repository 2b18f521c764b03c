"""Eigenvalue solve of the improved GmGM (FP64).

Test infrastructure only (see ``oracle/__init__``).

With the eigenvectors fixed by Theorem 1, the negative log-likelihood in the
eigenvalues (times 2, constants dropped) is

    f(Lam) = sum_l E_l . Lam_l  -  sum_gamma sum_{grid of gamma} log s,
    s(idx) = sum_{l in gamma} lam_{l, idx_l},

whose gradient is  g_l,i = E_l,i - sum_{gamma containing l} sum_{other idx} 1/s
(the Proposition on the eigenvalue gradient, and its elementwise form in the
existence lemma of the appendix "Existence and uniqueness").  f is convex.
The feasible set is the box Lam_l >= eps_l of that lemma (reading of
Assumption 4: the *smallest* eigenvalue is bounded below).

``solve_newton`` is a projected Newton method for box constraints
(Bertsekas, "Projected Newton methods for optimization problems with simple
constraints", SIAM J. Control Optim. 1982): nearly-active coordinates take a
diagonally scaled gradient step, the free ones a Newton step with the dense
Hessian H = d^2 f (entries sums of 1/s^2), and an Armijo search runs along the
projection arc.  It is deliberately a different algorithm from the GPU's.

``solve_alg1`` is the paper's own iteration (Algorithm 1): start at 1/E,
step Lam <- Lam - (mu/2) g, decrease mu while the step leaves the box.

Gauge (the diagonal shift of the appendix "Identifiability"): for one
modality, f(Lam + c) = f(Lam) + sum_l c_l tr(E_l) for shifts with
sum_l c_l = 0.  If all traces are equal the shift is flat and a convention
fixes it (every axis but the first has its smallest eigenvalue at eps);
otherwise f decreases along a shift until the box stops it, so the box fixes
the gauge.
"""

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg


@dataclass
class KSProblem:
    """Eigenvalue problem: per-axis spectra E_l and the modalities (tuples of
    axis indices, in tensor order) whose Kronecker-sum grids enter f."""
    E: list
    modalities: list = None
    eps: list = None
    r: list = field(init=False)
    off: np.ndarray = field(init=False)

    def __post_init__(self):
        self.E = [np.asarray(e, dtype=np.float64) for e in self.E]
        if self.modalities is None:
            self.modalities = [tuple(range(len(self.E)))]
        self.modalities = [tuple(m) for m in self.modalities]
        self.r = [len(e) for e in self.E]
        self.off = np.concatenate([[0], np.cumsum(self.r)])
        if self.eps is None:
            self.eps = default_eps(self.E, self.modalities)
        self.eps = [float(e) for e in self.eps]

    @property
    def n(self):
        return int(self.off[-1])

    def split(self, x):
        return [x[self.off[a]:self.off[a + 1]] for a in range(len(self.E))]

    def lower(self):
        return np.concatenate([np.full(r, e) for r, e in zip(self.r, self.eps)])

    def e_all(self):
        return np.concatenate(self.E)


def default_eps(E, modalities, rel=1e-10):
    """eps_l = rel * max_grid s at the paper's start Lam^0 = 1/E (one value for
    every axis): the largest sum over a modality of max_i 1/E_l,i."""
    big = max(sum(1.0 / np.min(E[a]) for a in m) for m in modalities)
    return [rel * big] * len(E)


def init_inv_e(prob: KSProblem):
    """Algorithm 1's initialisation Lam^0 = 1/E, lifted onto the box."""
    return np.maximum(1.0 / prob.e_all(), prob.lower())


def grid(lams, axes):
    """s over one modality's grid: s[i0, i1, ...] = sum_p lam_{axes[p], i_p}."""
    s = 0.0
    k = len(axes)
    for p, a in enumerate(axes):
        shape = [1] * k
        shape[p] = -1
        s = s + lams[a].reshape(shape)
    return s


def objective(x, prob: KSProblem):
    lams = prob.split(x)
    f = float(np.dot(prob.e_all(), x))
    for m in prob.modalities:
        s = grid(lams, m)
        if np.any(s <= 0):
            return np.inf
        f -= float(np.sum(np.log(s)))
    return f


def gradient(x, prob: KSProblem):
    lams = prob.split(x)
    g = [e.copy() for e in prob.E]
    for m in prob.modalities:
        inv = 1.0 / grid(lams, m)
        k = len(m)
        for p, a in enumerate(m):
            others = tuple(q for q in range(k) if q != p)
            g[a] -= inv.sum(axis=others) if others else inv
    return np.concatenate(g)


def hessian(x, prob: KSProblem):
    lams = prob.split(x)
    h = np.zeros((prob.n, prob.n))
    for m in prob.modalities:
        w = grid(lams, m) ** -2
        k = len(m)
        for p, a in enumerate(m):
            others = tuple(q for q in range(k) if q != p)
            d = w.sum(axis=others) if others else w
            sl = slice(prob.off[a], prob.off[a + 1])
            h[sl, sl] += np.diag(d)
            for q in range(p + 1, k):
                b = m[q]
                rest = tuple(t for t in range(k) if t not in (p, q))
                blk = w.sum(axis=rest) if rest else w
                sb = slice(prob.off[b], prob.off[b + 1])
                h[sl, sb] += blk
                h[sb, sl] += blk.T
    return h


def projected_gradient(x, g, lo):
    """KKT residual of the box problem: g on free coordinates, min(g, 0) on
    coordinates at their bound."""
    return np.where(x > lo, g, np.minimum(g, 0.0))


def rel_kkt(x, prob: KSProblem, g=None):
    """max_i |P(g)_i| / E_i, the relative projected-KKT residual."""
    if g is None:
        g = gradient(x, prob)
    return float(np.max(np.abs(projected_gradient(x, g, prob.lower())) / prob.e_all()))


@dataclass
class SolveInfo:
    iterations: int
    rel_kkt: float
    objective: float
    n_active: int
    converged: bool


def solve_newton(prob: KSProblem, x0=None, tol=1e-12, max_iter=300, sigma=1e-4,
                 gauge=True):
    """Projected Newton (Bertsekas 1982) on the box Lam >= eps.  Returns
    (x, SolveInfo); x is the concatenation of the per-axis Lam_l."""
    lo = prob.lower()
    x = init_inv_e(prob) if x0 is None else np.maximum(np.asarray(x0, np.float64), lo)
    f = objective(x, prob)
    if not np.isfinite(f):
        raise ValueError("infeasible start")
    it = 0
    g = gradient(x, prob)
    kkt = rel_kkt(x, prob, g)
    while kkt > tol and it < max_iter:
        it += 1
        h = hessian(x, prob)
        hd = np.diag(h).copy()
        # nearly-active: a diagonally scaled step would cross the bound
        act = (g > 0) & ((x - lo) <= g / hd)
        free = ~act
        d = np.zeros_like(x)
        d[act] = g[act] / hd[act]
        if np.any(free):
            hff = h[np.ix_(free, free)]
            sc = 1.0 / np.sqrt(np.diag(hff))
            a = hff * sc[:, None] * sc[None, :]
            a[np.diag_indices_from(a)] += 1e-13
            d[free] = sc * scipy.linalg.cho_solve(scipy.linalg.cho_factor(a), sc * g[free])
        alpha = 1.0
        accepted = False
        while alpha > 1e-30:
            xn = np.maximum(lo, x - alpha * d)
            fn = objective(xn, prob)
            dec = sigma * (alpha * np.dot(g[free], d[free]) + np.dot(g[act], x[act] - xn[act]))
            if fn <= f - dec:
                accepted = True
            elif np.isfinite(fn) and abs(fn - f) <= 1e-13 * (abs(f) + 1.0):
                # decrease below the rounding of f: accept if the KKT residual drops
                accepted = rel_kkt(xn, prob) < kkt
            if accepted:
                break
            alpha *= 0.5
        if not accepted:
            break
        x, f = xn, fn
        g = gradient(x, prob)
        kkt = rel_kkt(x, prob, g)
    if gauge:
        x = apply_gauge(x, prob)
    n_act = int(np.sum(x <= lo))
    return x, SolveInfo(it, rel_kkt(x, prob), objective(x, prob), n_act, kkt <= tol)


def traces_equal(prob: KSProblem, rtol=1e-9):
    t = np.array([e.sum() for e in prob.E])
    return bool(np.max(np.abs(t - t[0])) <= rtol * np.max(np.abs(t)))


def apply_gauge(x, prob: KSProblem, rtol=1e-9):
    """Gauge rule: with one modality and equal traces the shift is flat; move
    it so that every axis but the first has its minimum at eps, the first axis
    absorbing the opposite shift.  Otherwise the box already fixes the gauge
    and x is returned unchanged."""
    if len(prob.modalities) != 1 or not traces_equal(prob, rtol):
        return x
    lams = [l.copy() for l in prob.split(x)]
    for a in prob.modalities[0][1:]:
        c = prob.eps[a] - lams[a].min()
        lams[a] += c
        lams[prob.modalities[0][0]] -= c
    return np.concatenate(lams)


def solve_alg1(prob: KSProblem, tol=1e-8, max_iter=200000, mu0=1.0):
    """The paper's Algorithm 1 eigenvalue loop: Lam^0 = 1/E, mu = 1,
    Lam <- Lam - (mu/2)(E - sb-trace of the Kronecker-sum inverse).
    "Decrease mu if needed" is read as: halve mu while the step leaves the box
    or (a safeguard the paper leaves implicit) does not decrease f; "not
    converged" as rel_kkt > tol."""
    lo = prob.lower()
    x = init_inv_e(prob)
    f = objective(x, prob)
    mu = mu0
    it = 0
    g = gradient(x, prob)
    while rel_kkt(x, prob, g) > tol and it < max_iter:
        it += 1
        while True:
            xn = x - 0.5 * mu * g
            fn = objective(xn, prob) if np.all(xn >= lo) else np.inf
            if fn <= f:
                break
            mu *= 0.5
            if mu < 1e-300:
                return apply_gauge(x, prob), it
        x, f = xn, fn
        g = gradient(x, prob)
    return apply_gauge(x, prob), it


def two_axis_problem(e_rows, e_cols, eps=None):
    return KSProblem([e_rows, e_cols], [(0, 1)], eps)
