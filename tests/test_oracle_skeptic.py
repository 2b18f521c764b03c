"""Pins of the rank-based statistics oracle (oracle/skeptic.py) against the
paper's worked example and properties that hold for any data."""

import json
import os

import numpy as np
from scipy.special import ndtri

from oracle import skeptic as osk

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "skeptic_worked_example.json")


def _rng(seed):
    return np.random.default_rng(seed)


def test_worked_example_of_the_sparsity_appendix():
    g = json.load(open(GOLDEN))
    x = np.array(g["data"], dtype=np.float64)
    assert np.array_equal(osk.min_ranks(x), np.array(g["ranks"]))
    z = osk.normal_scores(x)
    assert np.max(np.abs(z - np.array(g["scores_2dp"]))) <= 0.005 + 1e-12
    zs = osk.zero_scores(x)
    assert np.max(np.abs(zs - np.array(g["zero_shift_2dp"]))) <= 0.005 + 1e-12
    # the sparse part of the decomposition keeps exactly the input's zeros
    sparse = z - zs[:, None]
    assert np.array_equal(sparse == 0.0, x == 0.0)


def test_min_ranks_against_counting():
    # ties in abundance (values 0..4): rank = 1 + number of strictly smaller entries
    x = _rng(1).integers(0, 5, size=(7, 23)).astype(np.float64)
    got = osk.min_ranks(x)
    for i in range(x.shape[0]):
        for j in range(x.shape[1]):
            assert got[i, j] == 1 + sum(1 for v in x[i] if v < x[i, j])


def test_scores_invariant_under_increasing_maps():
    # only the order inside a row matters (the copula assumption's point)
    x = _rng(2).standard_normal((9, 40))
    x[x < -0.5] = 0.0  # ties
    z = osk.normal_scores(x)
    for f in (lambda a: np.exp(a / 3.0), lambda a: a ** 3 + a, lambda a: 5.0 * a - 2.0):
        assert np.array_equal(osk.normal_scores(f(x)), z)


def test_rows_of_distinct_values_map_to_the_normal_quantiles():
    n = 31
    x = _rng(3).permuted(np.tile(np.arange(n, dtype=np.float64), (4, 1)), axis=1)
    z = osk.normal_scores(x)
    q = ndtri(np.arange(1, n + 1) / (n + 1.0))
    for row in z:
        assert np.array_equal(np.sort(row), q)
        assert abs(row.sum()) <= 1e-12  # quantiles symmetric about 1/2
    # the Gram's diagonal is then the same closed form for every row
    s = osk.skeptic_gram(x, 0)
    np.testing.assert_allclose(np.diag(s), np.sum(q * q), rtol=1e-14)


def test_zero_scores_match_the_zeros_of_every_row():
    x = _rng(4).poisson(0.4, size=(12, 50)).astype(np.float64)
    x[3] = 1.0 + np.arange(50)  # a row without zeros
    z = osk.normal_scores(x)
    zs = osk.zero_scores(x)
    for i in range(x.shape[0]):
        zero = x[i] == 0.0
        if zero.any():
            assert np.all(z[i][zero] == zs[i])
        else:
            assert zs[i] == 0.0


def test_skeptic_gram_is_per_axis_and_psd():
    t = _rng(5).poisson(1.5, size=(6, 8, 5)).astype(np.float64)
    for axis in range(3):
        s = osk.skeptic_gram(t, axis)
        assert s.shape == (t.shape[axis],) * 2
        assert np.array_equal(s, s.T)
        assert np.linalg.eigvalsh(s).min() >= -1e-10 * np.abs(s).max()
        # elementwise increasing transforms of the tensor leave it unchanged
        assert np.array_equal(osk.skeptic_gram(np.log1p(t), axis), s)
