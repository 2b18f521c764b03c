"""Pins of the oracle's Gram and spectra against definitions and invariants."""

import numpy as np
import pytest

from oracle.gram import gram, gram_multimodal, log1p_centre, log1p_col_means, matricize
from oracle.spectra import dual_lift, top_eigh, two_axis_spectra
from synth import planted_c1


def test_gram_matches_outer_product_loop():
    # Notation section: S_l = mat_l[X] mat_l[X]^T; brute force as a sum of
    # outer products of the matricisation's columns.
    rng = np.random.default_rng(1)
    x = rng.standard_normal((5, 4))
    s_cols = np.zeros((4, 4))
    s_rows = np.zeros((5, 5))
    for i in range(5):
        for a in range(4):
            for b in range(4):
                s_cols[a, b] += x[i, a] * x[i, b]
    for j in range(4):
        for a in range(5):
            for b in range(5):
                s_rows[a, b] += x[a, j] * x[b, j]
    np.testing.assert_allclose(gram(x, 1), s_cols, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(gram(x, 0), s_rows, rtol=1e-14, atol=1e-14)


def test_tensor_gram_trace_is_squared_norm_on_every_axis():
    rng = np.random.default_rng(2)
    t = rng.standard_normal((3, 4, 5))
    for ax in range(3):
        m = matricize(t, ax)
        assert m.shape == (t.shape[ax], t.size // t.shape[ax])
        np.testing.assert_allclose(np.trace(gram(t, ax)), np.sum(t * t), rtol=1e-13)
    # middle axis: slices X[a] (4 x 5); S_1 = sum_a X[a] X[a]^T
    s1 = sum(t[a] @ t[a].T for a in range(3))
    np.testing.assert_allclose(gram(t, 1), s1, rtol=1e-13, atol=1e-13)


def test_multimodal_gram_is_gram_of_concatenation():
    # Section "Algorithm": sum_gamma S_l^gamma = [mat_l D^1 ... mat_l D^G][...]^T
    rng = np.random.default_rng(3)
    x1 = rng.standard_normal((6, 4))   # cells x genes
    x2 = rng.standard_normal((6, 3))   # cells x peaks
    s = gram_multimodal([x1, x2], [("c", "g"), ("c", "p")], "c")
    cat = np.concatenate([x1, x2], axis=1)
    np.testing.assert_allclose(s, cat @ cat.T, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(gram_multimodal([x1, x2], [("c", "g"), ("c", "p")], "g"),
                               x1.T @ x1, rtol=1e-13)


def test_log1p_centre():
    c = np.array([[0, 1, 3], [2, 0, 0], [0, 0, 7]], dtype=np.float64)
    x = log1p_centre(c)
    np.testing.assert_allclose(x.mean(axis=0), 0, atol=1e-15)
    raw = np.log(1 + c)
    np.testing.assert_allclose(x + raw.mean(axis=0), raw, rtol=1e-15)


def test_log1p_col_means_closed_forms_and_row_blocks():
    # column 0 constant 4 -> log 5; column 1 one 1 in every 4 rows -> log(2)/4;
    # column 2 the counts 0..n-1 -> log(n!)/n (Python's lgamma), any blocking
    import math
    n = 1000
    c = np.zeros((n, 3), dtype=np.float32)
    c[:, 0] = 4
    c[::4, 1] = 1
    c[:, 2] = np.arange(n)
    want = [math.log(5.0), math.log(2.0) / 4, math.lgamma(n + 1) / n]
    for size in (n, 1, 7, 256):
        got = log1p_col_means((c[i:i + size] for i in range(0, n, size)), threads=3)
        np.testing.assert_allclose(got, want, rtol=1e-13)


def test_top_eigh_invariants():
    rng = np.random.default_rng(4)
    a = rng.standard_normal((30, 12))
    s = a.T @ a
    e, w = top_eigh(s, 12)
    assert np.all(np.diff(e) <= 0)
    np.testing.assert_allclose(s @ w, w * e[None, :], atol=1e-10 * e[0])
    np.testing.assert_allclose(w.T @ w, np.eye(12), atol=1e-13)
    # same spectrum as the characteristic roots found independently
    np.testing.assert_allclose(np.sort(e), np.sort(np.linalg.eigvals(s).real), rtol=1e-10)


def test_dual_lift_gives_left_singular_vectors():
    # Theorem 1 applied to the row axis: the lifted U are orthonormal
    # eigenvectors of X X^T with the same nonzero spectrum, and
    # X = U diag(sqrt E) W^T at full rank.
    x, _, _ = planted_c1()
    e_r, u, e_c, w = two_axis_spectra(x, 100, 100)
    np.testing.assert_allclose(e_r, e_c)
    np.testing.assert_allclose(u.T @ u, np.eye(100), atol=1e-10)
    srow = x @ x.T
    np.testing.assert_allclose(srow @ u, u * e_r[None, :], atol=1e-9 * e_r[0])
    np.testing.assert_allclose((u * np.sqrt(e_r)[None, :]) @ w.T, x, atol=1e-10)
    # truncated lift: top-r only
    e5, w5 = top_eigh(x.T @ x, 5)
    u5 = dual_lift(x, w5, e5)
    np.testing.assert_allclose(u5.T @ u5, np.eye(5), atol=1e-12)
    ev_rows = np.sort(np.linalg.eigvalsh(srow))[::-1][:5]
    np.testing.assert_allclose(e5, ev_rows, rtol=1e-10)


@pytest.mark.parametrize("block", [1, 7, 64, 1000])
def test_centred_gram_and_lift_over_row_blocks(block):
    # The row-blocked forms used at a million cells equal the plain
    # definitions: the Gram of log1p_centre(counts) and the dual lift of it,
    # whatever the blocking (a dropped rank-one term or a mean over the wrong
    # count would change every entry)
    from oracle.gram import log1p_centred_gram_blocks
    from oracle.spectra import dual_lift_blocks
    rng = np.random.default_rng(41)
    c = rng.poisson(rng.gamma(0.5, 2.0, size=(1, 9)), size=(120, 9)).astype(np.float32)
    c[:, 4] = 3.0  # a constant column: centred to exactly zero
    x = log1p_centre(c)
    ref = gram(x, 1)
    chunks = lambda: (c[i:i + block] for i in range(0, c.shape[0], block))
    s, mu, n = log1p_centred_gram_blocks(chunks())
    assert n == 120
    np.testing.assert_allclose(mu, np.log1p(c.astype(np.float64)).mean(axis=0), rtol=1e-14)
    np.testing.assert_allclose(s, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert np.all(np.abs(s[4]) <= 1e-12 * np.abs(ref).max())
    e, w = top_eigh(ref, 3)
    u = dual_lift_blocks(chunks(), mu, w, e)
    np.testing.assert_allclose(u, dual_lift(x, w, e), rtol=0, atol=1e-12)
    np.testing.assert_allclose(u.T @ u, np.eye(3), atol=1e-10)
