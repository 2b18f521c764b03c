"""Learned warm start of the eigenvalue solve (binding + training utilities).

The network and its training run in the library's CUDA kernels
(gmgm_warmstart_* / gmgm_mlp_*); this module marshals tensors, draws the
initial parameters and generates training pairs by running the method itself
(Gram, spectra, cold-start solve) on seeded synthetic problems.
"""

import ctypes
import os

import numpy as np
import torch

from . import _lib as L
from .api import _ptr, eigsolve, gram, handle, preprocess, spectra

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "warmstart_mlp.npz")


def init_params(seed=0, device="cuda"):
    """He-initialised parameters (FP32, flat, the ABI's layout), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for nout, nin in ((L.MLP_HIDDEN, L.MLP_IN), (L.MLP_HIDDEN, L.MLP_HIDDEN), (L.MLP_OUT, L.MLP_HIDDEN)):
        parts.append(rng.standard_normal((nout, nin)) * np.sqrt(2.0 / nin))
        parts.append(np.zeros(nout))
    p = np.concatenate([x.ravel() for x in parts]).astype(np.float32)
    assert p.size == L.MLP_PARAMS
    return torch.from_numpy(p).to(device)


def features(E0, E1, h=None):
    h = h or handle(E0.device)
    out = torch.empty(L.MLP_IN, dtype=torch.float32, device=E0.device)
    h.check(h.lib.gmgm_warmstart_features(h.h, _ptr(E0), E0.numel(), _ptr(E1), E1.numel(), _ptr(out)))
    return out


def targets(E0, E1, lam0, lam1, h=None):
    h = h or handle(E0.device)
    out = torch.empty(L.MLP_OUT, dtype=torch.float32, device=E0.device)
    h.check(h.lib.gmgm_warmstart_targets(h.h, _ptr(E0), E0.numel(), _ptr(E1), E1.numel(), _ptr(lam0),
                                         _ptr(lam1), _ptr(out)))
    return out


def forward(params, feats, h=None):
    h = h or handle(params.device)
    feats = feats.reshape(-1, L.MLP_IN).contiguous()
    out = torch.empty(feats.shape[0], L.MLP_OUT, dtype=torch.float32, device=params.device)
    h.check(h.lib.gmgm_mlp_forward(h.h, _ptr(params), _ptr(feats), feats.shape[0], _ptr(out)))
    return out


def loss_grad(params, feats, tgts, h=None):
    h = h or handle(params.device)
    feats = feats.reshape(-1, L.MLP_IN).contiguous()
    tgts = tgts.reshape(-1, L.MLP_OUT).contiguous()
    g = torch.empty_like(params)
    loss = ctypes.c_float()
    h.check(h.lib.gmgm_mlp_loss_grad(h.h, _ptr(params), _ptr(feats), _ptr(tgts), feats.shape[0], _ptr(g),
                                     ctypes.byref(loss)))
    return float(loss.value), g


def train(params, feats, tgts, steps=2000, batch=64, lr=1e-3, seed=0, adam=None, h=None):
    """Adam on the GPU; returns (final mini-batch loss, adam state)."""
    h = h or handle(params.device)
    feats = feats.reshape(-1, L.MLP_IN).contiguous()
    tgts = tgts.reshape(-1, L.MLP_OUT).contiguous()
    if adam is None:
        adam = torch.zeros(2 * L.MLP_PARAMS, dtype=torch.float32, device=params.device)
    o = L.TrainOpts(steps, batch, lr, 0.9, 0.999, 1e-8, seed)
    loss = ctypes.c_float()
    h.check(h.lib.gmgm_warmstart_train(h.h, _ptr(params), _ptr(adam), _ptr(feats), _ptr(tgts), feats.shape[0],
                                       ctypes.byref(o), ctypes.byref(loss)))
    return float(loss.value), adam


def infer(params, E0, E1, eps=0.0, h=None):
    """Predicted starting eigenvalues for a two-axis problem."""
    h = h or handle(E0.device)
    l0 = torch.empty_like(E0)
    l1 = torch.empty_like(E1)
    h.check(h.lib.gmgm_warmstart_infer(h.h, _ptr(params), _ptr(E0), E0.numel(), _ptr(E1), E1.numel(), eps,
                                       _ptr(l0), _ptr(l1)))
    return l0, l1


def method_problem(seed, device, cells=None, genes=None, r_cells=None, cell_range=(1000, 20000),
                   gene_range=(100, 600)):
    """One synthetic scRNA-like problem through the method's first steps on
    the GPU: returns (E_cells, E_genes) for the eigenvalue solve."""
    from synth import scrna_counts
    rng = np.random.default_rng(seed)
    cells = cells or int(np.exp(rng.uniform(np.log(cell_range[0]), np.log(cell_range[1]))))
    genes = genes or int(np.exp(rng.uniform(np.log(gene_range[0]), np.log(gene_range[1]))))
    # the full gene spectrum needs X of full column rank: at least twice as
    # many cells as genes (with fewer cells most gene eigenvalues are zero
    # and the box problem has no bounded optimum)
    genes = min(genes, cells // 2)
    r_cells = r_cells or int(rng.integers(8, min(100, genes // 2)))
    clusters = int(rng.integers(4, 40))
    counts = scrna_counts(cells, genes, clusters, seed=int(seed), device=device)
    x, _, _, _ = preprocess(counts, split=False)
    S = gram(x)
    e, _ = spectra(S, genes, vectors=False)
    return e[:r_cells].contiguous(), e.contiguous()


def method_pairs(n, seed=0, device="cuda", tol=1e-9, deadline=None, skipped=None, **ranges):
    """Up to n (features, targets) pairs: the method's own cold-start
    solutions of seeded synthetic problems (stops early at `deadline`, a
    time.time() value, if given).  Problems whose solve did not reach `tol`
    are left out (and listed in `skipped` if a list is given)."""
    import time
    F, T = [], []
    for i in range(n):
        if deadline is not None and time.time() > deadline:
            break
        e0, e1 = method_problem(seed * 100003 + i, device, **ranges)
        (l0, l1), st = eigsolve([e0, e1], [(0, 1)], tol=tol)
        if st["status"] != 0:
            if skipped is not None:
                skipped.append({"problem": i, "cells_rank": int(e0.numel()), "genes": int(e1.numel()), **st})
            continue
        F.append(features(e0, e1))
        T.append(targets(e0, e1, l0, l1))
    return torch.stack(F), torch.stack(T)


def save(params, path=WEIGHTS):
    np.savez_compressed(path, params=params.detach().cpu().numpy())


def load(device="cuda", path=WEIGHTS):
    if not os.path.exists(path):
        return None
    return torch.from_numpy(np.load(path)["params"]).to(device)
