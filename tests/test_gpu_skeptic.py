"""GPU parity of the rank-based statistics (the Nonparanormal Skeptic in its
COCA form) against the FP64 oracle: ranks bit-exact, scores within FP32
rounding, on the appendix's worked example, ragged shapes with heavy ties,
rows and columns with values beyond the kernels' bins, and the 1M-cell
workload's count recipe at 100,000 cells; invalid input sets the device
status bit."""

import json
import os

import numpy as np
import pytest
import torch

from oracle import skeptic as osk
from synth import scrna_counts

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "skeptic_worked_example.json")


@pytest.fixture(scope="module")
def g(cuda_dev):
    import paper_2407_19892_gb300 as pkg
    pkg.load()
    return pkg


def _ref(counts, axis):
    """Oracle ranks and scores along the axis (the oracle ranks rows)."""
    m = counts if axis == 0 else counts.T
    rk, z = osk.min_ranks(m), osk.normal_scores(m)
    return (rk, z) if axis == 0 else (rk.T, z.T)


def _check(g, counts, axis, dev):
    c = torch.from_numpy(np.ascontiguousarray(counts, dtype=np.float32)).to(dev)
    z, hi, lo, ld_t, rk = g.skeptic(c, axis, z=True, planes=True, ranks=True)
    h = g.handle(dev)
    assert h.device_status() == 0
    ref_r, ref_z = _ref(counts.astype(np.float64), axis)
    assert np.array_equal(rk.cpu().numpy(), ref_r)
    zg = z.cpu().numpy()
    np.testing.assert_allclose(zg, ref_z.astype(np.float32), rtol=2.4e-7, atol=1e-30)
    # the planes are the BF16 split of Z^T (zero beyond the rows)
    n = counts.shape[0]
    zt = (hi.float() + lo.float()).cpu().numpy()
    assert np.all(zt[:, n:] == 0)
    np.testing.assert_allclose(zt[:, :n], zg.T, rtol=2 ** -16, atol=0)
    return zg


def test_worked_example_of_the_sparsity_appendix(g, cuda_dev):
    # the appendix ranks its rows with negative entries; the GPU path takes
    # counts, so the example is shifted by +3 (ranks depend only on order)
    ex = json.load(open(GOLDEN))
    x = np.array(ex["data"], dtype=np.float64) + 3.0
    c = torch.from_numpy(x.astype(np.float32)).to(cuda_dev)
    z, _, _, _, rk = g.skeptic(c, g.AXIS_ROWS, planes=False, ranks=True)
    assert np.array_equal(rk.cpu().numpy(), np.array(ex["ranks"]))
    assert np.max(np.abs(z.cpu().numpy() - np.array(ex["scores_2dp"]))) <= 0.005 + 1e-7


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("n,p,lam", [(300, 77, 0.4), (1031, 129, 3.0), (64, 2000, 0.7), (5, 3, 1.0)])
def test_ranks_and_scores_match_the_oracle(g, cuda_dev, axis, n, p, lam):
    rng = np.random.default_rng(n * 7 + p + axis)
    counts = rng.poisson(lam, size=(n, p)).astype(np.float64)
    _check(g, counts, axis, cuda_dev)


@pytest.mark.parametrize("axis", [0, 1])
def test_values_beyond_the_bins(g, cuda_dev, axis):
    # rows (columns) mixing small counts with values of 1,000-100,000 and
    # ties among the large ones: the ROWS kernel's large-value path and the
    # COLS kernel's wide histograms
    rng = np.random.default_rng(50 + axis)
    counts = rng.poisson(2.0, size=(400, 300)).astype(np.float64)
    big = rng.random(counts.shape) < 0.05
    counts[big] = rng.choice([1023, 1024, 1025, 5000, 5000, 99999], size=big.sum())
    counts[7] = 2000.0  # an all-tied row
    counts[:, 11] = 0.0  # an all-zero column
    _check(g, counts, axis, cuda_dev)


@pytest.mark.parametrize("axis", [0, 1])
def test_scrna_counts_100k_cells(g, cuda_dev, axis):
    n, p = 100_000, 2000
    counts = scrna_counts(n, p, 20, seed=20240731)
    c = counts.to(cuda_dev)
    z, _, _, _, rk = g.skeptic(c, axis, planes=False, ranks=True)
    assert g.handle(cuda_dev).device_status() == 0
    rng = np.random.default_rng(9)
    cn = counts.numpy().astype(np.float64)
    if axis == 0:
        sel = rng.choice(n, 200, replace=False)
        ref_r, ref_z = _ref(cn[sel], 0)
        got_r, got_z = rk.cpu().numpy()[sel], z.cpu().numpy()[sel]
    else:
        sel = rng.choice(p, 40, replace=False)
        ref_r, ref_z = _ref(cn[:, sel], 1)
        got_r, got_z = rk.cpu().numpy()[:, sel], z.cpu().numpy()[:, sel]
    assert np.array_equal(got_r, ref_r)
    np.testing.assert_allclose(got_z, ref_z.astype(np.float32), rtol=2.4e-7, atol=1e-30)


@pytest.mark.parametrize("bad", [-1.0, 0.5, float("nan"), float("inf"), 2.0 ** 25])
@pytest.mark.parametrize("axis", [0, 1])
def test_invalid_counts_set_the_status_bit(g, cuda_dev, bad, axis):
    c = torch.ones(50, 20, device=cuda_dev)
    c[13, 4] = bad
    g.skeptic(c, axis, planes=False)
    assert g.handle(cuda_dev).device_status() == 0x20


def test_argument_errors(g, cuda_dev):
    c = torch.ones(10, 4, device=cuda_dev)
    h = g.handle(cuda_dev)
    with pytest.raises(g.GmgmError):  # no output
        h.check(h.lib.gmgm_skeptic(h.h, 10, 4, c.data_ptr(), 4, 0, None, 0, None, None, 0, None, 0))
    with pytest.raises(g.GmgmError):  # bad axis
        g.skeptic(c, 2)
    with pytest.raises(g.GmgmError):  # planes along ROWS need z_out
        hi = torch.empty(4, 64, dtype=torch.bfloat16, device=cuda_dev)
        h.check(h.lib.gmgm_skeptic(h.h, 10, 4, c.data_ptr(), 4, 0, None, 0, hi.data_ptr(), hi.data_ptr(), 64,
                                   None, 0))


def test_skeptic_fit_matches_the_oracle(g, cuda_dev):
    # the two-axis fit on rank-based statistics: each axis' Gram from its own
    # normal scores (genes ranked over cells, cells ranked over genes)
    from oracle.recon import topk_gap, topk_rows
    from oracle.solve import solve_newton, two_axis_problem
    from oracle.spectra import dual_lift, top_eigh
    n, p, r, k = 3000, 200, 15, 10
    counts = scrna_counts(n, p, 6, seed=20240802).numpy().astype(np.float64)
    res = g.fit_two_axis_skeptic(torch.from_numpy(counts.astype(np.float32)).to(cuda_dev), r, k, k)
    zc = osk.normal_scores(counts)          # cells ranked over genes
    zg = osk.normal_scores(counts.T)        # genes ranked over cells
    e_c, w_c = top_eigh(zc.T @ zc, r)
    e_g, _ = top_eigh(zg @ zg.T, p)
    np.testing.assert_allclose(res.e_rows.cpu().numpy(), e_c, rtol=5e-5)
    np.testing.assert_allclose(res.e_cols.cpu().numpy(), e_g, rtol=0, atol=5e-5 * e_g[0])
    lam, info = solve_newton(two_axis_problem(e_c, e_g))
    sr = lam[:r][:, None] + lam[r:][None, :]
    sg = res.lam_rows.cpu().numpy()[:, None] + res.lam_cols.cpu().numpy()[None, :]
    assert np.max(np.abs(sg - sr) / sr) <= 1e-4
    # the lifted cell vectors: U = Z_c W diag(E)^-1/2 (signs free)
    U = res.v_rows.cpu().numpy()
    ref = dual_lift(zc, w_c, e_c)
    sign = np.sign(np.sum(U * ref, axis=0))
    assert np.max(np.abs(U - ref * sign[None, :])) <= 1e-4 * np.abs(ref).max()
    # the cell network stage-wise on its own vectors
    lr = res.lam_rows.cpu().numpy()
    V = U.astype(np.float64)
    ri, _ = topk_rows(V, lr, k)
    gap = topk_gap(V, lr, k)
    idx = res.idx_rows.cpu().numpy()
    ok = gap > 1e-5
    assert np.array_equal(np.sort(idx[ok], 1), np.sort(ri[ok], 1)) and ok.mean() > 0.5
