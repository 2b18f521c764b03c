"""Pins of the warm-start reference network and its features."""

import numpy as np

from oracle import mlp


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(31)
    p = rng.standard_normal(mlp.n_params()) * 0.05
    x = rng.standard_normal((5, mlp.N_IN))
    t = rng.standard_normal((5, mlp.N_OUT))
    loss, g = mlp.loss_and_grad(p, x, t)
    idx = rng.choice(len(p), 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss_and_grad(p + e, x, t)[0] - mlp.loss_and_grad(p - e, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * (1 + abs(g[i]))


def test_forward_is_the_layer_formula():
    # a network whose layers are identity blocks reproduces ReLU(x) padded
    p = np.zeros(mlp.n_params())
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p)
    sizes = [W1.size, b1.size, W2.size, b2.size, W3.size, b3.size]
    o = np.cumsum([0] + sizes)
    eye1 = np.zeros((mlp.HIDDEN, mlp.N_IN)); eye1[:mlp.N_IN, :mlp.N_IN] = np.eye(mlp.N_IN)
    p[o[0]:o[1]] = eye1.ravel()
    p[o[2]:o[3]] = np.eye(mlp.HIDDEN).ravel()
    eye3 = np.zeros((mlp.N_OUT, mlp.HIDDEN)); eye3[:, :mlp.N_OUT] = np.eye(mlp.N_OUT)
    p[o[4]:o[5]] = eye3.ravel()
    x = np.random.default_rng(1).standard_normal((3, mlp.N_IN))
    y, _ = mlp.forward(p, x)
    np.testing.assert_allclose(y, np.maximum(x, 0)[:, :mlp.N_OUT])


def test_features_targets_expand_round_trip():
    # features of a geometric spectrum: its log-quantiles are a straight line;
    # expanding the targets of lam returns lam at the quantile positions
    e0 = np.geomspace(100.0, 1.0, 64)
    e1 = np.geomspace(50.0, 0.5, 200)
    f = mlp.features(e0, e1)
    assert f.shape == (mlp.N_IN,)
    np.testing.assert_allclose(np.diff(f[:64]), np.diff(f[:64])[0], rtol=1e-10)
    lam0 = 3.0 / e0
    lam1 = np.full(200, 0.25)
    t = mlp.targets(e0, e1, lam0, lam1)
    np.testing.assert_allclose(t[:64], np.log(3.0))
    l0, l1 = mlp.expand(t, e0, e1)
    np.testing.assert_allclose(l0, lam0, rtol=1e-12)
    # axis 1: log(lam E) is linear in the rank, so interpolation is exact at
    # the 64 quantile positions and close in between
    np.testing.assert_allclose(l1, lam1, rtol=2e-3)
