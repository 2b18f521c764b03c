"""Pins of the oracle's recomposition + per-row top-k."""

import heapq

import numpy as np
import pytest

from oracle import recon
from oracle.recon import recompose, topk_gap, topk_rows
from oracle.fit import fit_two_axis
from synth import planted_c1


def _heap_topk(psi, k):
    """Independent brute force: pure-Python heap over (|v|, -j)."""
    out = []
    for i in range(psi.shape[0]):
        h = []
        for j in range(psi.shape[1]):
            if j == i:
                continue
            key = (abs(psi[i, j]), -j)
            if len(h) < k:
                heapq.heappush(h, key)
            elif key > h[0]:
                heapq.heapreplace(h, key)
        best = sorted(h, reverse=True)
        out.append([-jj for _, jj in best])
    return np.array(out)


def test_planted_sparse_matrix_is_recovered_from_its_eigenpairs():
    # Recompose V diag(lam) V^T from the eigendecomposition of a known sparse
    # symmetric matrix with distinct off-diagonal magnitudes: the per-row
    # top-k must be read off the planted nonzeros.
    rng = np.random.default_rng(13)
    d, k = 40, 3
    psi = np.zeros((d, d))
    for i in range(d):
        for t, off in enumerate((1, 2, 5)):
            j = (i + off) % d
            w = (0.5 + 0.1 * t + 1e-3 * i) * (-1) ** (i + t)
            psi[i, j] = psi[j, i] = w
    np.fill_diagonal(psi, np.abs(psi).sum(1) + 1)
    lam, v = np.linalg.eigh(psi)
    idx, val = topk_rows(v, lam, k)
    for i in range(d):
        a = np.abs(psi[i]).copy(); a[i] = -1
        expect = np.lexsort((np.arange(d), -a))[:k]
        assert list(idx[i]) == list(expect)
        np.testing.assert_allclose(val[i], psi[i, expect], atol=1e-12)


def test_topk_matches_heap_brute_force():
    rng = np.random.default_rng(14)
    v = rng.standard_normal((60, 7))
    lam = rng.uniform(-1, 3, 7)
    idx, val = topk_rows(v, lam, 5, block=16)
    psi = recompose(v, lam)
    assert np.array_equal(idx, _heap_topk(psi, 5))
    np.testing.assert_allclose(val, np.take_along_axis(psi, idx, 1), rtol=1e-14)


def test_ties_break_by_lower_column_and_diagonal_excluded():
    # V = I_4 with equal lam: Psi = 2 I, every off-diagonal is 0 (a 3-way tie).
    v = np.eye(4)
    idx, val = topk_rows(v, np.full(4, 2.0), 2)
    assert idx.tolist() == [[1, 2], [0, 2], [0, 1], [0, 1]]
    assert np.all(val == 0)
    gap = topk_gap(v, np.full(4, 2.0), 2)
    assert np.all(gap == 0)


def _planted_gap_matrix():
    """A dense symmetric 16 x 16 matrix whose rows have known, distinct
    off-diagonal magnitudes (random signs, a dominant diagonal that must
    never count), with row 0 planted so that its 3rd and 4th magnitudes are
    1e-5 apart relative to the 3rd, and row 1 so that its 3rd-4th gap
    differs from its 4th-5th gap and from the gap over the 4th."""
    rng = np.random.default_rng(31)
    d = 16
    psi = np.zeros((d, d))
    mags = rng.permutation(np.linspace(0.05, 0.95, d * (d - 1) // 2))
    iu = np.triu_indices(d, 1)
    psi[iu] = mags * rng.choice([-1.0, 1.0], size=mags.size)
    # row 0: magnitudes 2.0, 1.5, 1.2, 1.2 (1 - 1e-5), then the rest below 1
    for j, m in zip((5, 9, 2, 13), (2.0, -1.5, 1.2, -1.2 * (1.0 - 1e-5))):
        psi[0, j] = m
    # row 1: 3.0, 2.5, 2.0, 1.6, 1.5: gap(k=3) = 0.2, gap over the 4th 0.25,
    # gap(4th, 5th) = 0.0625
    for j, m in zip((7, 3, 12, 15, 6), (3.0, 2.5, -2.0, 1.6, -1.5)):
        psi[1, j] = m
    psi = np.triu(psi, 1)
    psi = psi + psi.T
    np.fill_diagonal(psi, 50.0 + np.arange(d))
    return psi


def _sorted_gap(row, i, k):
    """Brute force: the full sorted list of a row's off-diagonal magnitudes."""
    a = sorted((abs(x) for j, x in enumerate(row) if j != i), reverse=True)
    return (a[k - 1] - a[k]) / a[k - 1]


def test_topk_gap_on_planted_magnitudes():
    psi = _planted_gap_matrix()
    lam, v = np.linalg.eigh(psi)
    k = 3
    gap = topk_gap(v, lam, k, block=5)
    # the recomposition is exact to ~1e-14 of the diagonal; gaps to 1e-11
    for i in range(psi.shape[0]):
        assert abs(gap[i] - _sorted_gap(psi[i], i, k)) < 1e-11
    assert abs(gap[0] - 1e-5) < 1e-11
    assert abs(gap[1] - 0.2) < 1e-11
    # an off-by-one (4th vs 5th) or the wrong denominator (the 4th) would give
    assert abs(gap[1] - 0.0625) > 0.1 and abs(gap[1] - 0.25) > 0.04
    # sampled rows agree with the full computation
    sub = topk_gap(v, lam, k, rows=[1, 0, 15])
    np.testing.assert_allclose(sub, gap[[1, 0, 15]], rtol=0, atol=1e-12)
    # k = d - 1 has no (k+1)-th entry: an infinite gap
    assert np.all(np.isinf(topk_gap(v, lam, psi.shape[0] - 1)))


def test_topk_gap_random_rows_against_full_sort():
    rng = np.random.default_rng(32)
    v = rng.standard_normal((70, 9))
    lam = rng.uniform(-2.0, 3.0, 9)
    psi = recompose(v, lam)
    for k in (1, 4, 10):
        gap = topk_gap(v, lam, k, block=16)
        ref = np.array([_sorted_gap(psi[i], i, k) for i in range(70)])
        np.testing.assert_allclose(gap, ref, rtol=1e-9, atol=1e-13)


def test_sampled_rows_equal_full_rows():
    rng = np.random.default_rng(15)
    v = rng.standard_normal((50, 4))
    lam = rng.uniform(0.1, 1, 4)
    full_i, full_v = topk_rows(v, lam, 4)
    rows = np.array([3, 17, 49, 0])
    si, sv = topk_rows(v, lam, 4, rows=rows)
    assert np.array_equal(si, full_i[rows])
    np.testing.assert_allclose(sv, full_v[rows])


def test_planted_recovery_sanity_c1():
    # Sanity bound, not parity: the strongest genes-axis edges of the fit on
    # the planted 200 x 100 draw overlap the planted ER graph far above chance.
    x, psi1, psi2 = planted_c1()
    fit = fit_two_axis(x, 100, 100, 10, 10)
    idx, _ = fit.topk_cols
    true = np.abs(psi2) > 0
    np.fill_diagonal(true, False)
    hits = sum(true[i, j] for i in range(100) for j in idx[i, :2])
    prec = hits / (2 * 100)
    density = true.sum() / (100 * 99)
    assert prec > 2 * density  # about 3x chance from one 200 x 100 draw


# ---- global top-n (the paper's heap of n_l edges) -----------------------------

def _brute_topn(V, lam, n):
    psi = recon.recompose(V, lam)
    d = psi.shape[0]
    edges = [(-abs(psi[i, j]), i, j, psi[i, j]) for i in range(d) for j in range(i + 1, d)]
    edges.sort()
    top = edges[:n]
    return (np.array([e[1] for e in top]), np.array([e[2] for e in top]), np.array([e[3] for e in top]))


@pytest.mark.parametrize("block", [1, 4, 256])
def test_topn_edges_is_the_sorted_pair_list(block):
    rng = np.random.default_rng(11)
    V = rng.standard_normal((25, 4))
    lam = rng.uniform(0.5, 2.0, 4)
    i, j, v = recon.topn_edges(V, lam, 37, block=block)
    bi, bj, bv = _brute_topn(V, lam, 37)
    assert np.array_equal(i, bi) and np.array_equal(j, bj)
    np.testing.assert_allclose(v, bv, rtol=1e-13, atol=1e-13)


def test_topn_edges_orders_ties_by_pair():
    # duplicated rows: equal magnitudes, ordered by (i, j)
    rng = np.random.default_rng(12)
    V = np.repeat(rng.standard_normal((6, 3)), 3, axis=0)
    lam = rng.uniform(0.5, 1.5, 3)
    i, j, v = recon.topn_edges(V, lam, 40)
    bi, bj, bv = _brute_topn(V, lam, 40)
    assert np.array_equal(i, bi) and np.array_equal(j, bj)


def test_topn_from_row_lists_certified_equals_global():
    rng = np.random.default_rng(13)
    V = rng.standard_normal((80, 6))
    lam = rng.uniform(0.5, 2.0, 6)
    idx, val = recon.topk_rows(V, lam, 10)
    i, j, v, ok = recon.topn_from_row_lists(idx, val, 40)
    assert ok
    gi, gj, gv = recon.topn_edges(V, lam, 40)
    assert np.array_equal(i, gi) and np.array_equal(j, gj)
    np.testing.assert_allclose(v, gv, rtol=1e-12)


def test_topn_from_row_lists_refuses_a_clique_its_lists_cannot_hold():
    # a 12-node clique of strong edges: with 5 slots per row at most 60 of its
    # 66 edges reach the union, so the derivation must not claim the top 66.
    # With 11 slots every clique edge is listed, but a clique row's list is
    # then all strong and could hide a 12th: still not certified.  With 12
    # slots each clique row shows one weak entry and it is certified
    rng = np.random.default_rng(14)
    d = 40
    M = 10.0 * np.eye(d) + 0.01 * rng.standard_normal((d, d))
    M[:12, :12] += 5.0 + 0.1 * rng.standard_normal((12, 12))
    M = 0.5 * (M + M.T)
    lam, V = np.linalg.eigh(M)
    idx, val = recon.topk_rows(V, lam, 5)
    *_, ok = recon.topn_from_row_lists(idx, val, 66)
    assert not ok
    idx, val = recon.topk_rows(V, lam, 11)
    *_, ok = recon.topn_from_row_lists(idx, val, 66)
    assert not ok
    idx, val = recon.topk_rows(V, lam, 12)
    i, j, v, ok = recon.topn_from_row_lists(idx, val, 66)
    assert ok
    gi, gj, _ = recon.topn_edges(V, lam, 66)
    assert np.array_equal(i, gi) and np.array_equal(j, gj)
    assert np.all(i < 12) and np.all(j < 12)
