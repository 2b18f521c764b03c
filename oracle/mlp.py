"""FP64 reference of the warm-start network and its features (test infrastructure).

Test infrastructure only (see ``oracle/__init__``).  The paper has no learned
component: Algorithm 1 starts the eigenvalue solve at Lam^0 = 1/E.  The warm
start replaces that start by a prediction; it is judged by the plain solve,
which always runs to the same tolerance from it.

Definitions (mirrored by the GPU kernels):

* features of a two-axis problem (E_0, E_1 descending, ranks r_0, r_1):
  for each axis l and k = 0..63, the linear interpolation of log E_l at
  position k/63 * (r_l - 1), minus log(mean E_l); then four extras:
  log(r_0)/8, log(r_1)/8, log tr E_0 - log tr E_1, log E_0[0] - log E_1[0].
* targets of a solved problem: for each axis, the interpolation of
  log(lam_l,i * E_l,i) at the same 64 positions.
* network: 132 -> 256 -> 256 -> 128, ReLU on the hidden layers, linear output;
  loss = mean squared error over outputs and samples.
* inverse map of a prediction y (64 per axis): for rank index i, the
  interpolation of y at position i/(r-1) * 63, lam_i = exp(.) / E_i.
"""

import numpy as np

NQ = 64
N_IN = 2 * NQ + 4
N_OUT = 2 * NQ
HIDDEN = 256


def _interp(vals, r, nq=NQ):
    pos = np.arange(nq) / (nq - 1) * (r - 1)
    lo = np.floor(pos).astype(int)
    hi = np.minimum(lo + 1, r - 1)
    fr = pos - lo
    return vals[lo] * (1 - fr) + vals[hi] * fr


def features(e0, e1):
    e0 = np.asarray(e0, np.float64)
    e1 = np.asarray(e1, np.float64)
    f = []
    for e in (e0, e1):
        f.append(_interp(np.log(e), len(e)) - np.log(np.mean(e)))
    extra = [np.log(len(e0)) / 8, np.log(len(e1)) / 8,
             np.log(e0.sum()) - np.log(e1.sum()), np.log(e0[0]) - np.log(e1[0])]
    return np.concatenate(f + [np.array(extra)])


def targets(e0, e1, lam0, lam1):
    out = []
    for e, l in ((e0, lam0), (e1, lam1)):
        out.append(_interp(np.log(np.asarray(l, np.float64) * np.asarray(e, np.float64)), len(e)))
    return np.concatenate(out)


def expand(y, e0, e1):
    """Per-axis eigenvalues from a prediction y (128 values)."""
    out = []
    for a, e in enumerate((e0, e1)):
        e = np.asarray(e, np.float64)
        r = len(e)
        q = y[a * NQ:(a + 1) * NQ]
        pos = np.arange(r) / max(r - 1, 1) * (NQ - 1)
        lo = np.floor(pos).astype(int)
        hi = np.minimum(lo + 1, NQ - 1)
        fr = pos - lo
        out.append(np.exp(q[lo] * (1 - fr) + q[hi] * fr) / e)
    return out


def unpack(params, n_in=N_IN, h=HIDDEN, n_out=N_OUT):
    """Flat parameter vector -> (W1, b1, W2, b2, W3, b3), W as [out, in]."""
    sizes = [(h, n_in), (h,), (h, h), (h,), (n_out, h), (n_out,)]
    out, o = [], 0
    for s in sizes:
        n = int(np.prod(s))
        out.append(np.asarray(params[o:o + n], np.float64).reshape(s))
        o += n
    return out


def n_params(n_in=N_IN, h=HIDDEN, n_out=N_OUT):
    return h * n_in + h + h * h + h + n_out * h + n_out


def forward(params, x):
    W1, b1, W2, b2, W3, b3 = unpack(params)
    z1 = x @ W1.T + b1
    a1 = np.maximum(z1, 0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0)
    return a2 @ W3.T + b3, (x, z1, a1, z2, a2)


def loss_and_grad(params, x, t):
    """MSE (mean over samples and outputs) and its gradient (flat, FP64)."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    y, (x, z1, a1, z2, a2) = forward(params, x)
    n = y.size
    loss = float(np.sum((y - t) ** 2) / n)
    dy = 2.0 * (y - t) / n
    gW3 = dy.T @ a2
    gb3 = dy.sum(0)
    da2 = dy @ W3
    dz2 = da2 * (z2 > 0)
    gW2 = dz2.T @ a1
    gb2 = dz2.sum(0)
    da1 = dz2 @ W2
    dz1 = da1 * (z1 > 0)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(0)
    return loss, np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3)])
