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


# ---- cone bound for skipping column tiles ---------------------------------------

def test_cone_bound_bounds_every_column_of_the_tile():
    rng = np.random.default_rng(21)
    for trial in range(50):
        r = int(rng.integers(2, 12))
        centre = rng.standard_normal(r)
        spread = 10.0 ** rng.uniform(-3, 0.5)
        b = centre[None, :] + spread * rng.standard_normal((64, r))
        b *= rng.choice([-1.0, 1.0], size=(64, 1)) * rng.uniform(0.2, 3.0, size=(64, 1))
        a = rng.standard_normal((40, r)) * rng.uniform(0.1, 10.0, size=(40, 1))
        c, s, bmax = recon.tile_cone(b)
        exact = np.max(np.abs(a @ b.T), axis=1)
        assert np.all(exact <= cone_bound_tol(recon.cone_bound(a, c, s, bmax)))


def cone_bound_tol(x):
    return x * (1.0 + 1e-12) + 1e-300


def test_cone_bound_is_attained_for_aligned_and_boundary_columns():
    # two columns of norm 2 at angle t: the cone's centre is their bisector,
    # sin(theta) = sin(t / 2).  A row along the bisector meets the first term
    # (|a . c| = 1, exact 2 cos(t / 2)); a row orthogonal to the bisector in
    # their plane meets the bound exactly (2 sin(t / 2) both)
    r, t = 6, 0.3
    b = np.zeros((2, r))
    b[0, 0] = 2.0
    b[1, :2] = 2.0 * np.cos(t), 2.0 * np.sin(t)
    c, s, bmax = recon.tile_cone(b)
    assert bmax == 2.0 and abs(s - np.sin(t / 2)) < 1e-12
    a = np.zeros((2, r))
    a[0, :2] = np.cos(t / 2), np.sin(t / 2)
    a[1, :2] = -np.sin(t / 2), np.cos(t / 2)
    exact = np.max(np.abs(a @ b.T), axis=1)
    bound = recon.cone_bound(a, c, s, bmax)
    assert abs(exact[0] - 2.0 * np.cos(t / 2)) < 1e-12 and bound[0] >= exact[0]
    assert abs(exact[1] - 2.0 * np.sin(t / 2)) < 1e-12 and abs(bound[1] - exact[1]) < 1e-12


def test_cone_bound_rules_out_tiles_of_other_directions():
    # columns clustered around e_0, rows along e_1: the bound is small, while
    # Cauchy-Schwarz alone (||a|| max ||b||) would keep the tile
    rng = np.random.default_rng(22)
    r = 10
    e0 = np.zeros(r); e0[0] = 1.0
    b = e0[None, :] + 0.05 * rng.standard_normal((256, r))
    a = np.zeros((1, r)); a[0, 1] = 1.0
    c, s, bmax = recon.tile_cone(b)
    bound = recon.cone_bound(a, c, s, bmax)[0]
    assert bound < 0.35 * bmax * np.linalg.norm(a)
    assert np.max(np.abs(a @ b.T)) <= bound
