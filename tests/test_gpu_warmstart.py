"""Learned warm start: GPU features / forward / gradient against the FP64
reference network, GPU training, and what the trained network saves the
eigenvalue solve (which always runs to the same tolerance)."""

import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from oracle import solve as osv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws(cuda_dev):
    from paper_2407_19892_gb300 import build
    build.build()
    from paper_2407_19892_gb300 import warmstart
    return warmstart


def _spectra(rng, r0, r1):
    e0 = np.sort(np.exp(rng.normal(2.0, 1.0, r0)))[::-1].copy()
    e1 = np.sort(np.exp(rng.normal(1.0, 0.7, r1)))[::-1].copy()
    return e0, e1


def test_features_and_targets_match_reference(ws, cuda_dev):
    rng = np.random.default_rng(41)
    for r0, r1 in ((7, 300), (64, 64), (130, 2000)):
        e0, e1 = _spectra(rng, r0, r1)
        t0, t1 = torch.from_numpy(e0).to(cuda_dev), torch.from_numpy(e1).to(cuda_dev)
        f = ws.features(t0, t1).cpu().numpy()
        np.testing.assert_allclose(f, omlp.features(e0, e1), rtol=1e-5, atol=1e-5)
        l0 = rng.uniform(0.5, 2.0, r0) / e0
        l1 = rng.uniform(0.5, 2.0, r1) / e1
        t = ws.targets(t0, t1, torch.from_numpy(l0).to(cuda_dev), torch.from_numpy(l1).to(cuda_dev)).cpu().numpy()
        np.testing.assert_allclose(t, omlp.targets(e0, e1, l0, l1), rtol=1e-5, atol=1e-5)


def test_forward_and_gradient_match_reference(ws, cuda_dev):
    p = ws.init_params(3, cuda_dev)
    rng = np.random.default_rng(42)
    x = rng.standard_normal((37, omlp.N_IN)).astype(np.float32)
    t = rng.standard_normal((37, omlp.N_OUT)).astype(np.float32)
    X, T = torch.from_numpy(x).to(cuda_dev), torch.from_numpy(t).to(cuda_dev)
    y = ws.forward(p, X).cpu().numpy()
    pr = p.double().cpu().numpy()
    y_ref, _ = omlp.forward(pr, x.astype(np.float64))
    np.testing.assert_allclose(y, y_ref, rtol=1e-4, atol=1e-4 * np.abs(y_ref).max())
    loss, g = ws.loss_grad(p, X, T)
    loss_ref, g_ref = omlp.loss_and_grad(pr, x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    g = g.double().cpu().numpy()
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)


def test_training_and_warm_start_save_iterations(ws, cuda_dev):
    import paper_2407_19892_gb300 as pkg
    F, T = ws.method_pairs(96, seed=1, device=cuda_dev)
    assert F.shape[0] >= 80
    p = ws.init_params(0, cuda_dev)
    loss0, _ = ws.loss_grad(p, F, T)
    loss1, _ = ws.train(p, F, T, steps=1500, batch=32, lr=1e-3, seed=7)
    loss_all, _ = ws.loss_grad(p, F, T)
    assert loss_all < 0.1 * loss0, (loss0, loss1, loss_all)
    cold, warm = [], []
    for i in range(8):  # held-out problems
        e0, e1 = ws.method_problem(987654 + i, cuda_dev)
        (a0, a1), st_c = pkg.eigsolve([e0, e1], [(0, 1)], tol=1e-9)
        i0, i1 = ws.infer(p, e0, e1)
        (b0, b1), st_w = pkg.eigsolve([e0, e1], [(0, 1)], tol=1e-9, init=[i0, i1])
        assert st_c["status"] == 0 and st_w["status"] == 0
        s_c = (a0[:, None] + a1[None, :]).cpu().numpy()
        s_w = (b0[:, None] + b1[None, :]).cpu().numpy()
        assert np.max(np.abs(s_c - s_w) / s_c) <= 1e-6  # same optimum either way
        cold.append(st_c["newton_iters"])
        warm.append(st_w["newton_iters"])
    assert np.mean(warm) < np.mean(cold), (cold, warm)
