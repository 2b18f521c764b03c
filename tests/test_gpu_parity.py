"""GPU parity: every C-ABI entry point against the FP64 oracle on the same
seeded inputs (sizes that span several tiles and a ragged tail)."""

import numpy as np
import pytest
import torch

from oracle import gram as og
from oracle import recon as orc
from oracle import solve as osv
from oracle import spectra as osp
from synth import planted_c1, scrna_counts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g(cuda_dev):
    import paper_2407_19892_gb300 as pkg
    from paper_2407_19892_gb300 import build
    build.build()
    return pkg


def _rng(seed):
    return np.random.default_rng(seed)


# ---- preprocessing ---------------------------------------------------------

@pytest.mark.parametrize("n,p", [(1000, 130), (4097, 64), (2, 1)])
def test_preprocess_matches_oracle(g, cuda_dev, n, p):
    counts = scrna_counts(n, max(p, 2), 5, seed=11)[:, :p].contiguous()
    x, hi, lo, ld_t = g.preprocess(counts.to(cuda_dev), split=True)
    ref = og.log1p_centre(counts.numpy())
    np.testing.assert_allclose(x.cpu().numpy(), ref, atol=2e-6 * max(1.0, np.abs(ref).max()))
    xt = (hi.float() + lo.float()).cpu().numpy()
    assert xt.shape == (p, ld_t) and ld_t % 64 == 0
    np.testing.assert_allclose(xt[:, :n], x.cpu().numpy().T, atol=1e-4 * max(1.0, np.abs(ref).max()))
    assert np.all(xt[:, n:] == 0)
    # planes only (no FP32 X written): the same planes, bit for bit
    x2, hi2, lo2, ld2 = g.preprocess(counts.to(cuda_dev), split=True, x_out=False)
    assert x2 is None and ld2 == ld_t
    assert torch.equal(hi2, hi) and torch.equal(lo2, lo)


# ---- Gram ------------------------------------------------------------------

@pytest.mark.parametrize("n,p", [(5000, 200), (777, 65), (64, 1)])
def test_gram_fp32_cols(g, cuda_dev, n, p):
    x = _rng(1).standard_normal((n, p)).astype(np.float32)
    S = g.gram(torch.from_numpy(x).to(cuda_dev), g.SIDE_COLS, g.FP32).cpu().numpy()
    ref = og.gram(x.astype(np.float64), 1)
    assert np.max(np.abs(S - ref)) <= 2e-6 * np.abs(ref).max()
    assert np.array_equal(S, S.T)


def _split_planes(x, dev):
    """BF16 hi/lo planes of X^T (p x ld_t, zero padded), as the preprocessing
    kernel lays them out."""
    n, p = x.shape
    ld_t = ((n + 63) // 64) * 64
    xt = torch.zeros(p, ld_t, dtype=torch.float32, device=dev)
    xt[:, :n] = torch.from_numpy(x).to(dev).T
    hi = xt.to(torch.bfloat16)
    lo = (xt - hi.float()).to(torch.bfloat16)
    return hi.contiguous(), lo.contiguous(), ld_t


@pytest.mark.parametrize("n,p", [(5000, 300), (20000, 2000), (70, 5), (9000, 129)])
def test_gram_tensor_core_3xbf16(g, cuda_dev, n, p):
    x = _rng(11 + p).standard_normal((n, p)).astype(np.float32)
    hi, lo, ld_t = _split_planes(x, cuda_dev)
    ref = og.gram(x.astype(np.float64), 1)
    S3 = g.gram(None, g.SIDE_COLS, g.BF16X3, xt_hi=hi, xt_lo=lo, ld_t=ld_t, rows=n, cols=p).cpu().numpy()
    err3 = np.max(np.abs(S3 - ref)) / np.abs(ref).max()
    assert err3 <= 2e-5, err3
    assert np.array_equal(S3, S3.T)
    S1 = g.gram(None, g.SIDE_COLS, g.BF16, xt_hi=hi, ld_t=ld_t, rows=n, cols=p).cpu().numpy()
    err1 = np.max(np.abs(S1 - ref)) / np.abs(ref).max()
    assert err1 <= 2e-2, err1
    assert err3 < err1


def test_gram_rows_and_tensor_axes(g, cuda_dev):
    t = _rng(2).standard_normal((7, 40, 33)).astype(np.float32)
    tt = torch.from_numpy(t).to(cuda_dev)
    s0 = g.gram(tt.reshape(7, 40 * 33), g.SIDE_ROWS, g.FP32).cpu().numpy()
    s1 = g.gram(tt, g.SIDE_ROWS, g.FP32).cpu().numpy()           # batch of 40 x 33 slices
    s2 = g.gram(tt.reshape(7 * 40, 33), g.SIDE_COLS, g.FP32).cpu().numpy()
    for ax, s in enumerate((s0, s1, s2)):
        ref = og.gram(t.astype(np.float64), ax)
        assert np.max(np.abs(s - ref)) <= 2e-6 * np.abs(ref).max(), ax


def test_gram_accumulate_is_multimodal_sum(g, cuda_dev):
    r = _rng(3)
    x1 = r.standard_normal((300, 50)).astype(np.float32)
    x2 = r.standard_normal((300, 70)).astype(np.float32)
    S = g.gram(torch.from_numpy(x1).to(cuda_dev), g.SIDE_ROWS, g.FP32)
    g.gram(torch.from_numpy(x2).to(cuda_dev), g.SIDE_ROWS, g.FP32, out=S, accumulate=True)
    ref = og.gram_multimodal([x1.astype(np.float64), x2.astype(np.float64)], [("c", "g"), ("c", "p")], "c")
    assert np.max(np.abs(S.cpu().numpy() - ref)) <= 2e-6 * np.abs(ref).max()


# ---- spectra -----------------------------------------------------------------

def _check_eig(S, ev, W, r):
    e_ref, w_ref = osp.top_eigh(S, r)
    scale = np.abs(e_ref).max()
    np.testing.assert_allclose(ev, e_ref, rtol=0, atol=1e-11 * scale)
    if W is not None:
        res = S @ W - W * ev[None, :]
        assert np.max(np.abs(res)) <= 1e-10 * scale
        assert np.max(np.abs(W.T @ W - np.eye(r))) <= 1e-8


@pytest.mark.parametrize("d,r", [(300, 300), (257, 17), (3, 3), (2, 1), (1, 1), (1000, 1000)])
def test_spectra_random_gram(g, cuda_dev, d, r):
    x = _rng(4).standard_normal((d + 50, d))
    S = x.T @ x
    ev, W = g.spectra(torch.from_numpy(S).to(cuda_dev), r)
    _check_eig(S, ev.cpu().numpy(), W.cpu().numpy(), r)


def test_spectra_degenerate_and_clustered(g, cuda_dev):
    # identity (one eigenvalue of multiplicity d) and a block of near-equal values
    d = 120
    S = np.eye(d) * 3.0
    ev, W = g.spectra(torch.from_numpy(S).to(cuda_dev), 40)
    _check_eig(S, ev.cpu().numpy(), W.cpu().numpy(), 40)
    q, _ = np.linalg.qr(_rng(5).standard_normal((d, d)))
    lam = np.linspace(1.0, 2.0, d)
    lam[:10] = 5.0 + 1e-13 * np.arange(10)
    S = (q * lam) @ q.T
    S = 0.5 * (S + S.T)
    ev, W = g.spectra(torch.from_numpy(S).to(cuda_dev), 30)
    _check_eig(S, ev.cpu().numpy(), W.cpu().numpy(), 30)


@pytest.mark.parametrize("case", ["logspace", "scaled_up", "scaled_down", "d4000"])
def test_spectra_range_and_scaling(g, cuda_dev, case):
    # the reduction runs in double-float on a power-of-two-scaled copy:
    # eigenvalues spread over twelve decades, Grams scaled by 2^+-100
    # (far outside the FP32 range before scaling) and a 4000 x 4000 Gram
    # must still match the oracle to FP64-like accuracy
    rng = _rng(12)
    if case == "logspace":
        d = 600
        q, _ = np.linalg.qr(rng.standard_normal((d, d)))
        S = (q * np.logspace(-6, 6, d)) @ q.T
    elif case == "d4000":
        d = 4000
        x = rng.standard_normal((d + 50, d))
        S = x.T @ x
    else:
        d = 500
        x = rng.standard_normal((d + 50, d))
        S = (x.T @ x) * (2.0 ** (100 if case == "scaled_up" else -100))
    S = 0.5 * (S + S.T)
    r = 40
    ev, W = g.spectra(torch.from_numpy(S).to(cuda_dev), d, rv=r)
    ev = ev.cpu().numpy()
    W = W.cpu().numpy()
    e_ref, _ = osp.top_eigh(S, d)
    scale = np.abs(e_ref).max()
    np.testing.assert_allclose(ev, e_ref, rtol=0, atol=1e-11 * scale)
    assert np.max(np.abs(S @ W - W * ev[None, :r])) <= 1e-10 * scale
    assert np.max(np.abs(W.T @ W - np.eye(r))) <= 1e-8


def test_lift_matches_oracle(g, cuda_dev):
    x, _, _ = planted_c1()
    x = (x - x.mean(0)).astype(np.float32)
    S = og.gram(x.astype(np.float64), 1)
    e, w = osp.top_eigh(S, 37)
    U = g.lift(torch.from_numpy(x).to(cuda_dev), torch.from_numpy(w).to(cuda_dev),
               torch.from_numpy(e).to(cuda_dev), 37).cpu().numpy()
    ref = osp.dual_lift(x.astype(np.float64), w, e)
    assert np.max(np.abs(U - ref)) <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("n,p,r", [(1000, 300, 50), (70001, 2000, 64), (257, 61, 7), (5000, 130, 33)])
def test_lift_tensor_core_from_planes(g, cuda_dev, n, p, r):
    # the 3xBF16 tensor-core lift from the BF16 planes of X^T (several
    # 256-cell blocks and 128-gene drains, ragged cells and genes) against the
    # oracle's FP64 lift of the same centred log1p matrix, and the FP32 form
    counts = scrna_counts(n, p, 8, seed=300 + n + r)
    x, hi, lo, ld_t = g.preprocess(counts.to(cuda_dev), split=True)
    x64 = og.log1p_centre(counts.numpy())
    e, w = osp.top_eigh(og.gram(x64, 1), r)
    W, E = torch.from_numpy(w).to(cuda_dev), torch.from_numpy(e).to(cuda_dev)
    U = g.lift(x, W, E, r, xt_hi=hi, xt_lo=lo, ld_t=ld_t).cpu().numpy()
    ref = osp.dual_lift(x64, w, e)
    assert np.max(np.abs(U - ref)) <= 1e-5 * np.abs(ref).max()
    U32 = g.lift(x, W, E, r).cpu().numpy()
    assert np.max(np.abs(U - U32)) <= 1e-5 * np.abs(ref).max()


# ---- eigenvalue solve ------------------------------------------------------------

def _sums(lams, mods):
    out = []
    for m in mods:
        s = osv.grid([np.asarray(l) for l in lams], m)
        out.append(np.asarray(s).ravel())
    return np.concatenate(out)


def _solve_case(g, cuda_dev, E, mods, tol=1e-9):
    prob = osv.KSProblem(E, mods)
    ref, info = osv.solve_newton(prob)
    lams, st = g.eigsolve([torch.from_numpy(e).to(cuda_dev) for e in E], mods, tol=tol)
    got = [l.cpu().numpy() for l in lams]
    assert st["status"] == 0, st
    assert st["rel_kkt"] <= 10 * tol, st
    a = _sums(got, mods)
    b = _sums(prob.split(ref), mods)
    err = np.max(np.abs(a - b) / np.abs(b))
    return err, st, got, prob


def test_eigsolve_full_rank_gauge(g, cuda_dev):
    x, _, _ = planted_c1()
    e_r, _, e_c, _ = osp.two_axis_spectra(x, 100, 100)
    err, st, got, prob = _solve_case(g, cuda_dev, [e_r, e_c], [(0, 1)])
    assert err <= 1e-7, err
    # gauge convention: min of the second axis at eps
    assert abs(got[1].min() - prob.eps[1]) <= 1e-12 * got[0].max()


@pytest.mark.parametrize("r1", [1, 10, 37])
def test_eigsolve_truncated_box(g, cuda_dev, r1):
    x, _, _ = planted_c1()
    e_r, _, e_c, _ = osp.two_axis_spectra(x, r1, 100)
    err, st, got, prob = _solve_case(g, cuda_dev, [e_r, e_c], [(0, 1)])
    assert err <= 1e-7, err
    assert st["n_active"] > 0


def test_eigsolve_scrna_like_spectrum(g, cuda_dev):
    counts = scrna_counts(4000, 300, 8, seed=21)
    x = og.log1p_centre(counts.numpy())
    e_all, _ = osp.top_eigh(x.T @ x, 300)
    err, st, _, _ = _solve_case(g, cuda_dev, [e_all[:40], e_all], [(0, 1)])
    assert err <= 1e-7, err


def test_eigsolve_three_axis_and_multimodal(g, cuda_dev):
    r = _rng(6)
    t = r.standard_normal((5, 7, 6))
    es = [osp.top_eigh(og.gram(t, a), t.shape[a])[0] for a in range(3)]
    err, st, _, _ = _solve_case(g, cuda_dev, es, [(0, 1, 2)])
    assert err <= 1e-7, err
    # two modalities sharing axis 0 (cells x genes, cells x peaks), truncated cells
    x1 = r.standard_normal((60, 20))
    x2 = r.standard_normal((60, 30))
    sc = og.gram_multimodal([x1, x2], [("c", "g"), ("c", "p")], "c")
    e_c = osp.top_eigh(sc, 15)[0]
    e_g = osp.top_eigh(x1.T @ x1, 20)[0]
    e_p = osp.top_eigh(x2.T @ x2, 30)[0]
    err, st, _, _ = _solve_case(g, cuda_dev, [e_c, e_g, e_p], [(0, 1), (0, 2)])
    assert err <= 1e-7, err


def test_eigsolve_three_axis_traces_equal_to_fp32_rounding(g, cuda_dev):
    # full-rank spectra of one tensor: equal traces in exact arithmetic; a
    # relative 1e-7 perturbation (spectra from FP32 Grams) must still give
    # the flat shift, a converged solve and the gauge convention
    r = _rng(7)
    t = r.standard_normal((6, 9, 8))
    es = [osp.top_eigh(og.gram(t, a), t.shape[a])[0] for a in range(3)]
    pert = [es[0] * (1 + 1e-7), es[1], es[2] * (1 - 8e-8)]
    lams, st = g.eigsolve([torch.from_numpy(e).to(cuda_dev) for e in pert], [(0, 1, 2)], tol=1e-10)
    assert st["status"] == 0 and st["rel_kkt"] <= 1e-10, st
    l = [x.cpu().numpy() for x in lams]
    from oracle.solve import KSProblem, solve_newton
    prob = KSProblem(es, [(0, 1, 2)])
    ref, _ = solve_newton(prob, tol=1e-12)
    rl = prob.split(ref)
    s = l[0][:, None, None] + l[1][None, :, None] + l[2][None, None, :]
    sr = rl[0][:, None, None] + rl[1][None, :, None] + rl[2][None, None, :]
    assert np.max(np.abs(s - sr) / sr) <= 1e-6
    for a in (1, 2):
        assert abs(l[a].min() - prob.eps[a]) <= 1e-6 * prob.eps[a]
    # with the tolerance off the perturbed traces count as different
    _, st_off = g.eigsolve([torch.from_numpy(e).to(cuda_dev) for e in pert], [(0, 1, 2)], tol=1e-10, trace_rtol=-1.0)
    assert st_off["status"] in (0, -5)


def test_eigsolve_warm_start_and_fp64_only(g, cuda_dev):
    x, _, _ = planted_c1()
    e_r, _, e_c, _ = osp.two_axis_spectra(x, 20, 100)
    E = [torch.from_numpy(e).to(cuda_dev) for e in (e_r, e_c)]
    lams, st = g.eigsolve(E, [(0, 1)], tol=1e-10, fp32_phase=False)
    assert st["status"] == 0 and st["rel_kkt"] <= 1e-9
    lams2, st2 = g.eigsolve(E, [(0, 1)], tol=1e-10, init=lams)
    assert st2["newton_iters"] <= 1
    for a, b in zip(lams, lams2):
        torch.testing.assert_close(a, b, rtol=1e-8, atol=0)


@pytest.mark.parametrize("bad,code", [(0.0, -6), (-1.0, -6), (float("nan"), -4), (float("inf"), -4)])
def test_eigsolve_rejects_nonpositive_or_nonfinite_E(g, cuda_dev, bad, code):
    # a zero eigenvalue (X without full rank on an axis) leaves f unbounded
    # below: no iteration runs, the outputs are NaN, the status says why
    x, _, _ = planted_c1()
    e_r, _, e_c, _ = osp.two_axis_spectra(x, 20, 100)
    e_c = e_c.copy()
    e_c[-1] = bad
    E = [torch.from_numpy(e).to(cuda_dev) for e in (e_r, e_c)]
    with pytest.raises(g.GmgmError) as ei:
        g.eigsolve(E, [(0, 1)])
    assert ei.value.code == code
    h = g.handle(cuda_dev)
    bits = h.device_status()
    assert bits & (0x4 if code == -6 else 0x1)
    # the handle stays usable: the same call on valid spectra converges
    e_c[-1] = e_c[-2] * 0.5
    E = [torch.from_numpy(e).to(cuda_dev) for e in (e_r, e_c)]
    lams, st = g.eigsolve(E, [(0, 1)])
    assert st["status"] == 0 and all(torch.isfinite(l).all() for l in lams)


# ---- top-k ------------------------------------------------------------------------

def _check_topk(V64, lam, k, idx, val, rows=None):
    """Stage-wise parity: the oracle's FP64 top-k of the same V, psi (of the
    given rows only, when ``rows`` is set; idx/val are then those rows')."""
    ref_i, ref_v = orc.topk_rows(V64, lam, k, rows=rows)
    gap = orc.topk_gap(V64, lam, k, rows=rows)
    ok = gap > 1e-5
    assert np.array_equal(np.sort(idx[ok], 1), np.sort(ref_i[ok], 1))
    # order inside the list follows the exact values
    mag = np.abs(ref_v[ok])
    distinct = np.all(np.diff(mag, axis=1) < -1e-12 * mag[:, :1], axis=1)
    assert np.array_equal(idx[ok][distinct], ref_i[ok][distinct])
    np.testing.assert_allclose(np.take_along_axis(val, np.argsort(idx, 1), 1)[ok],
                               np.take_along_axis(ref_v, np.argsort(ref_i, 1), 1)[ok].astype(np.float32),
                               rtol=1e-6, atol=1e-30)
    return ok.mean()


@pytest.mark.parametrize("d,r,k", [(1000, 50, 10), (517, 7, 32), (40, 3, 5), (20, 64, 19), (300, 200, 20)])
def test_topk_fp32_random(g, cuda_dev, d, r, k):
    rng = _rng(7 + d)
    V = rng.standard_normal((d, r)).astype(np.float32)
    lam = rng.uniform(0.1, 2.0, r)
    idx, val, st = g.topk_network(torch.from_numpy(V).to(cuda_dev), torch.from_numpy(lam).to(cuda_dev), k)
    frac = _check_topk(V.astype(np.float64), lam, k, idx.cpu().numpy(), val.cpu().numpy())
    assert frac > 0.9
    assert st["screen_err_ratio"] <= 1.0, st


@pytest.mark.parametrize("d,r,k", [(3000, 50, 10), (1000, 64, 20), (257, 7, 5), (100, 16, 32), (40, 3, 5)])
def test_topk_bf16_tensor_core_screen(g, cuda_dev, d, r, k):
    # tcgen05 screen + FP64 rescoring: exact FP64 top-k where the gap allows,
    # the screen inside its stated error bound, and most rows certified by
    # the tensor-core screen itself (a broken screen would flag every row).
    rng = _rng(100 + d)
    V = rng.standard_normal((d, r)).astype(np.float32)
    lam = rng.uniform(0.1, 2.0, r)
    idx, val, st = g.topk_network(torch.from_numpy(V).to(cuda_dev), torch.from_numpy(lam).to(cuda_dev), k,
                                  prec=g.BF16)
    frac = _check_topk(V.astype(np.float64), lam, k, idx.cpu().numpy(), val.cpu().numpy())
    assert frac > 0.9
    assert st["screen_err_ratio"] <= 1.0, st
    if d > 64 and k <= 20:  # with k near the 32 candidate slots no row can be certified
        assert st["rows_uncertified"] <= 0.5 * d, st


@pytest.mark.parametrize("clustered", [False, True])
def test_topk_bf16_long_sweep_sampled_rows(g, cuda_dev, clustered):
    # 40,000 columns: 157 B tiles per row block, long enough for the main
    # screen's sampling pass (threshold floor from every 16th tile); the
    # oracle's FP64 top-k of 500 sampled rows, and a valid list on every row.
    # Clustered rows (200 centroids + noise) put a row's strongest partners
    # in few columns, the case where a floor is most often too high for a
    # half's list to fill
    rng = _rng(41 + clustered)
    d, r, k = 40000, 50, 10
    if clustered:
        cent = rng.standard_normal((200, r))
        V = cent[rng.integers(0, 200, d)] + 0.3 * rng.standard_normal((d, r))
    else:
        V = rng.standard_normal((d, r))
    V = V.astype(np.float32)
    lam = rng.uniform(0.1, 2.0, r)
    idx, val, st = g.topk_network(torch.from_numpy(V).to(cuda_dev), torch.from_numpy(lam).to(cuda_dev), k,
                                  prec=g.BF16)
    idx, val = idx.cpu().numpy(), val.cpu().numpy()
    assert st["screen_err_ratio"] <= 1.0, st
    srt = np.sort(idx, 1)
    assert np.all(srt[:, 1:] != srt[:, :-1]) and np.all(idx >= 0) and np.all(idx < d)
    assert not np.any(idx == np.arange(d)[:, None])
    rows = np.sort(rng.choice(d, 500, replace=False))
    frac = _check_topk(V.astype(np.float64), lam, k, idx[rows], val[rows], rows=rows)
    assert frac > 0.9
    assert st["rows_exact"] <= d // 100, st


def test_topk_fp64_input_and_ties(g, cuda_dev):
    # duplicate rows give exact ties: lower column index first
    rng = _rng(8)
    base = rng.standard_normal((50, 6))
    V = np.repeat(base, 3, axis=0)
    lam = rng.uniform(0.5, 1.5, 6)
    idx, val, st = g.topk_network(torch.from_numpy(V).to(cuda_dev), torch.from_numpy(lam).to(cuda_dev), 4)
    ref_i, ref_v = orc.topk_rows(V, lam, 4)
    assert np.array_equal(idx.cpu().numpy(), ref_i)
    np.testing.assert_allclose(val.cpu().numpy(), ref_v.astype(np.float32), rtol=1e-6)


def test_topk_identity_all_zero_ties(g, cuda_dev):
    V = np.eye(40)
    lam = np.ones(40)
    idx, val, st = g.topk_network(torch.from_numpy(V).to(cuda_dev), torch.from_numpy(lam).to(cuda_dev), 3)
    ref_i, _ = orc.topk_rows(V, lam, 3)
    assert np.array_equal(idx.cpu().numpy(), ref_i)
    assert st["rows_uncertified"] == 40


def test_topk_bf16_repair_screen_certifies_near_ties(g, cuda_dev):
    # clustered rows (30 centroids + 2e-3 noise): neighbours inside a cluster
    # differ by far less than the BF16 screen's error bound, so most rows fail
    # its certification; the 3xBF16 repair screen (bound ~120x tighter)
    # certifies them, and the result is the exact FP64 top-k
    rng = _rng(31)
    d, r, k = 4000, 50, 10
    cent = rng.standard_normal((30, r))
    V = (cent[rng.integers(0, 30, d)] + 2e-3 * rng.standard_normal((d, r))).astype(np.float32)
    lam = rng.uniform(0.5, 2.0, r)
    idx, val, st = g.topk_network(torch.from_numpy(V).to(cuda_dev), torch.from_numpy(lam).to(cuda_dev), k,
                                  prec=g.BF16)
    frac = _check_topk(V.astype(np.float64), lam, k, idx.cpu().numpy(), val.cpu().numpy())
    assert frac > 0.5
    assert st["screen_err_ratio"] <= 1.0, st
    assert st["rows_uncertified"] > d // 4, st
    assert st["rows_exact"] <= st["rows_uncertified"] // 4, st


def _orthonormal(d, seed):
    q, _ = np.linalg.qr(_rng(seed).standard_normal((d, d)))
    return q


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_topk_ortho_split_of_clipped_eigenvalues(g, cuda_dev, prec):
    # full-rank axis with 250 of 300 eigenvalues at the box: the network of
    # c I + V diag(psi - c) V^T is that of the 50 free columns (the tensor
    # screen handles them at r = 50 for a BF16 request)
    d, k = 300, 10
    V = _orthonormal(d, 71)
    psi = np.full(d, 1e-3)
    free = _rng(72).choice(d, 50, replace=False)
    psi[free] = _rng(73).uniform(0.5, 2.0, 50)
    idx, val, st = g.topk_network(torch.from_numpy(V).to(cuda_dev), torch.from_numpy(psi).to(cuda_dev), k,
                                  g.FP32 if prec == "fp32" else g.BF16, ortho=True)
    frac = _check_topk(V, psi, k, idx.cpu().numpy(), val.cpu().numpy())
    assert frac > 0.9
    assert st["screen_err_ratio"] <= 1.0


def test_topk_ortho_all_at_the_minimum_is_all_ties(g, cuda_dev):
    # psi = c everywhere: Psi = c I, every off-diagonal entry is exactly 0 and
    # each row takes the k lowest columns j != i with value 0
    d, k = 257, 20
    V = _orthonormal(d, 74)
    psi = np.full(d, 3e-9)
    idx, val, st = g.topk_network(torch.from_numpy(V).to(cuda_dev), torch.from_numpy(psi).to(cuda_dev), k,
                                  ortho=True)
    want = np.array([[c if c < i else c + 1 for c in range(k)] for i in range(d)])
    assert np.array_equal(idx.cpu().numpy(), want)
    assert np.all(val.cpu().numpy() == 0.0)


def test_topk_argument_errors(g, cuda_dev):
    V = torch.zeros(10, 3, device=cuda_dev)
    psi = torch.ones(3, dtype=torch.float64, device=cuda_dev)
    with pytest.raises(g.GmgmError):
        g.topk_network(V, psi, 10)      # k >= d
    with pytest.raises(g.GmgmError):
        g.topk_network(V, psi, 33)      # k > 32
    with pytest.raises(g.GmgmError):
        g.topk_network(V, psi, 3, g.BF16X3)  # no split-product screen
    with pytest.raises(g.GmgmError):
        g.topk_network(V, psi, 3, ortho=True)  # the orthonormal split needs a square V
    with pytest.raises(g.GmgmError):
        g.topk_network(torch.zeros(100, 65, device=cuda_dev), torch.ones(65, dtype=torch.float64, device=cuda_dev),
                       3, g.BF16)       # tensor-core screen needs r <= 64


# ---- whole two-axis fit ---------------------------------------------------------------

def test_fit_two_axis_c1(g, cuda_dev):
    from oracle.fit import fit_two_axis as ofit
    x, _, _ = planted_c1()
    x = (x - x.mean(0)).astype(np.float32)
    res = g.fit_two_axis(torch.from_numpy(x).to(cuda_dev), 30, 100, 10, 10)
    ref = ofit(x.astype(np.float64), 30, 100, 10, 10)
    sg = res.lam_rows.cpu().numpy()[:, None] + res.lam_cols.cpu().numpy()[None, :]
    sr = ref.lam_rows[:, None] + ref.lam_cols[None, :]
    assert np.max(np.abs(sg - sr) / sr) <= 1e-4
    # the gene axis is at full rank: its network comes from the Gram (no
    # vectors returned); the stage-wise check uses FP64 eigenvectors of the
    # GPU's own Gram
    assert res.v_cols is None
    W = np.linalg.eigh(res.s_cols.cpu().numpy())[1][:, ::-1]
    for V, lam, k, idx, val in ((res.v_rows.double().cpu().numpy(), res.lam_rows, 10, res.idx_rows, res.val_rows),
                                (W, res.lam_cols, 10, res.idx_cols, res.val_cols)):
        _check_topk(V, lam.cpu().numpy(), k, idx.cpu().numpy(), val.cpu().numpy())


def test_fit_two_axis_truncated_gene_axis(g, cuda_dev):
    # both axes truncated: the gene vectors come from the spectra call
    from oracle.fit import fit_two_axis as ofit
    x, _, _ = planted_c1()
    x = (x - x.mean(0)).astype(np.float32)
    res = g.fit_two_axis(torch.from_numpy(x).to(cuda_dev), 30, 60, 10, 10)
    ref = ofit(x.astype(np.float64), 30, 60, 10, 10)
    sg = res.lam_rows.cpu().numpy()[:, None] + res.lam_cols.cpu().numpy()[None, :]
    sr = ref.lam_rows[:, None] + ref.lam_cols[None, :]
    assert np.max(np.abs(sg - sr) / sr) <= 1e-4
    assert res.v_cols.shape == (100, 60)
    _check_topk(res.v_cols.cpu().numpy(), res.lam_cols.cpu().numpy(), 10, res.idx_cols.cpu().numpy(),
                res.val_cols.cpu().numpy())


def test_topk_network_gram_matches_the_square_vectors(g, cuda_dev):
    # the network from the Gram equals the network of its full eigenvector
    # matrix (stage-wise, FP64 eigenvectors of the same S), with free
    # eigenvalues scattered over the spectrum and the rest at the minimum
    d, k = 220, 12
    A = _rng(81).standard_normal((400, d))
    S = A.T @ A
    psi = np.full(d, 2e-6)
    free = _rng(82).choice(d, 40, replace=False)
    psi[free] = _rng(83).uniform(1e-3, 1e-2, 40)
    idx, val, st = g.topk_network_gram(torch.from_numpy(S).to(cuda_dev), torch.from_numpy(psi).to(cuda_dev), k)
    W = np.linalg.eigh(S)[1][:, ::-1]
    frac = _check_topk(W, psi, k, idx.cpu().numpy(), val.cpu().numpy())
    assert frac > 0.9
    assert st["screen_err_ratio"] <= 1.0
    # every psi at the minimum: all ties
    idx, val, _ = g.topk_network_gram(torch.from_numpy(S).to(cuda_dev), torch.full((d,), 3.0, dtype=torch.float64,
                                                                                    device=cuda_dev), k)
    assert np.array_equal(idx.cpu().numpy()[:, 0], np.array([1] + [0] * (d - 1)))
    assert np.all(val.cpu().numpy() == 0.0)


def test_spectra_vectors_for_the_top_rv_only(g, cuda_dev):
    S = _rng(84).standard_normal((300, 300))
    S = S @ S.T
    ev_all, W_all = g.spectra(torch.from_numpy(S).to(cuda_dev), 300, rv=300)
    ev, W = g.spectra(torch.from_numpy(S).to(cuda_dev), 300, rv=25)
    assert W.shape == (300, 25)
    np.testing.assert_array_equal(ev.cpu().numpy(), ev_all.cpu().numpy())
    _check_eig(S, ev.cpu().numpy()[:25], W.cpu().numpy(), 25)
    ev0, W0 = g.spectra(torch.from_numpy(S).to(cuda_dev), 300, vectors=False)
    assert W0 is None
    np.testing.assert_array_equal(ev0.cpu().numpy(), ev_all.cpu().numpy())


@pytest.mark.parametrize("prec", ["FP32", "BF16"])
def test_topk_network_gram_2000_genes_every_eigenvalue_free(g, cuda_dev, prec):
    # The gene network of the 1M-cell workload's shape (d = 2000, k = 20)
    # with every psi distinct, so all 1999 eigenvectors above the minimum are
    # formed (tridiagonalisation, bisection, inverse iteration and the
    # back-transformation at full size) and the screen runs over r = 1999:
    # every row against the oracle's top-k of the FP64 eigenvectors of S
    d, k = 2000, 20
    rng = _rng(91)
    A = rng.standard_normal((5000, d)) * np.exp(rng.uniform(-2.0, 1.0, d))[None, :]
    S = A.T @ A
    w, W = np.linalg.eigh(S)
    w, W = w[::-1], W[:, ::-1]
    psi = 1.0 / w + rng.uniform(0.0, 1e-3, d) / w[0]
    idx, val, st = g.topk_network_gram(torch.from_numpy(S).to(cuda_dev), torch.from_numpy(psi).to(cuda_dev), k,
                                       getattr(g, prec))
    frac = _check_topk(W, psi, k, idx.cpu().numpy(), val.cpu().numpy())
    assert frac > 0.9
    assert st["screen_err_ratio"] <= 1.0


@pytest.mark.parametrize("prec", ["FP32", "BF16"])
def test_topk_network_rows_equals_the_rows_of_the_full_network(g, cuda_dev, prec):
    # a block of rows (what one rank of a row-sharded fit computes) is the
    # same rows of the whole network: the same certified lists and values
    rng = _rng(95)
    d, r, k = 3000, 50, 10
    V = torch.from_numpy(rng.standard_normal((d, r)).astype(np.float32)).to(cuda_dev)
    psi = torch.from_numpy(rng.uniform(0.1, 2.0, r)).to(cuda_dev)
    p = getattr(g, prec)
    idx, val, _ = g.topk_network(V, psi, k, p)
    for row0, m in ((0, 1000), (1000, 2000), (1234, 1), (2999, 1), (517, 700)):
        bi, bv, st = g.topk_network_rows(V, psi, k, row0, m, p)
        assert torch.equal(bi, idx[row0:row0 + m]) and torch.equal(bv, val[row0:row0 + m])
        assert st["screen_err_ratio"] <= 1.0
    with pytest.raises(g.GmgmError):
        g.topk_network_rows(V, psi, k, 2500, 501, p)


def test_topk_bf16_screen_counts_its_tiles(g, cuda_dev):
    # the screen reports the 128 x 256 tiles it multiplied: one dense sweep
    # (row blocks x column tiles) plus the sampling pass over every 16th
    # tile of each row block (the roofline is taken on this executed work)
    rng = _rng(62)
    d, r, k = 40000, 50, 10
    V = torch.from_numpy(rng.standard_normal((d, r)).astype(np.float32)).to(cuda_dev)
    lam = torch.from_numpy(rng.uniform(0.1, 2.0, r)).to(cuda_dev)
    _, _, st = g.topk_network(V, lam, k, prec=g.BF16)
    nrb, nt = (d + 127) // 128, (d + 255) // 256
    assert st["screen_tiles_dense"] == nrb * nt
    assert st["screen_tiles"] == nrb * (nt + (nt + 15) // 16), st
    _, _, st32 = g.topk_network(V, lam, k, prec=g.FP32)
    assert st32["screen_tiles"] == 0 and st32["screen_tiles_dense"] == 0


def test_eigsolve_grid_over_a_million_points_uses_every_sm(g, cuda_dev):
    # a 1100 x 1000 grid (1.1e6 points): the passes are split over all SMs
    # (cooperative launch); the result must equal the oracle's as for the
    # one-CTA solve
    rng = _rng(97)
    E = [np.sort(rng.uniform(0.5, 3.0, 1100))[::-1].copy(), np.sort(rng.uniform(0.2, 4.0, 1000))[::-1].copy()]
    err, st, got, prob = _solve_case(g, cuda_dev, E, [(0, 1)])
    assert err <= 1e-7, (err, st)
