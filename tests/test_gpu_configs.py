"""Parity at the other workloads' full sizes.

* 100,000 cells x 2,000 genes, plain FP32 form (FP32 SIMT Gram and screen),
  20 clusters, cell axis rank 100, full gene spectrum, k = 10: the FP64
  oracle runs the whole fit at this size (Gram, spectra, solve) and the
  networks are checked stage-wise on sampled rows.
* Multi-modal, 500,000 cells x (2,000 genes + 5,000 peaks) sharing the cell
  axis, BF16 tiles, cell axis rank 50, k = 10: checked on sampled Gram
  entries (FP64 from the counts), eigendecomposition and KKT properties,
  and the networks stage-wise on sampled rows.
"""

import numpy as np
import pytest
import torch

from oracle.fit import fit_two_axis as ofit
from oracle.gram import log1p_centre, log1p_col_means
from oracle.recon import topk_gap, topk_rows
from oracle.solve import KSProblem, rel_kkt
from synth import atac_binary, scrna_counts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_2407_19892_gb300 as g
    g.load()
    return g


def _sampled_rows_exact(V64, lam, k, rows, idx):
    """The FP64 top-k of the given rows of V diag(lam) V^T where it is
    determined (k-th/(k+1)-th gap above 1e-5 relative and the k-th magnitude
    above the FP64 rounding floor 1e-10 sqrt(Psi_ii max_j Psi_jj)); elsewhere
    k distinct off-diagonal columns reaching the k-th magnitude within that
    floor.  Returns the determined fraction."""
    ref_i, _ = topk_rows(V64, lam, k, rows=rows)
    gap = topk_gap(V64, lam, k, rows=rows)
    diag_max = float(np.max(np.einsum("ij,j,ij->i", V64, lam, V64)))
    psi = (V64[rows] * lam[None, :]) @ V64.T
    det = 0
    for t, i in enumerate(rows):
        a = np.abs(psi[t])
        floor = 1e-10 * np.sqrt(abs(psi[t, i]) * diag_max)
        a[i] = -np.inf
        kth = np.partition(a, -k)[-k]
        assert len(set(idx[t].tolist())) == k and i not in idx[t]
        assert np.all(a[idx[t]] >= kth - floor)
        if gap[t] > 1e-5 and kth > floor:
            det += 1
            assert np.array_equal(np.sort(idx[t]), np.sort(ref_i[t]))
    return det / len(rows)


def test_fp32_form_100k_cells(g, cuda_dev):
    n, p, r, k = 100_000, 2000, 100, 10
    counts = scrna_counts(n, p, 20, seed=20240729)
    x, _, _, _ = g.preprocess(counts.to(cuda_dev), split=False)
    res = g.fit_two_axis(x, r, p, k, k, gram_prec=g.FP32, topk_prec=g.FP32, tol=1e-9)
    ref = ofit(log1p_centre(counts.numpy()), r, p, k, k, sample_rows=np.arange(4))
    e = res.e_cols.cpu().numpy()
    np.testing.assert_allclose(e, ref.e_cols, rtol=0, atol=1e-5 * ref.e_cols[0])
    sg = res.lam_rows.cpu().numpy()[:, None] + res.lam_cols.cpu().numpy()[None, :]
    sr = ref.lam_rows[:, None] + ref.lam_cols[None, :]
    assert np.max(np.abs(sg - sr) / sr) <= 1e-4
    rows = np.sort(np.random.default_rng(3).choice(n, 64, replace=False))
    frac = _sampled_rows_exact(res.v_rows.double().cpu().numpy(), res.lam_rows.cpu().numpy(), k, rows,
                               res.idx_rows.cpu().numpy()[rows])
    assert frac > 0.5
    assert res.topk_rows_stats["screen_err_ratio"] <= 1.0
    W = np.linalg.eigh(res.s_cols.cpu().numpy())[1][:, ::-1]
    _sampled_rows_exact(W, res.lam_cols.cpu().numpy(), k, np.arange(p), res.idx_cols.cpu().numpy())


def test_multimodal_500k_cells(g, cuda_dev):
    n, pg, pp, r, k, cl = 500_000, 2000, 5000, 50, 10, 50
    c1, lab, _ = scrna_counts(n, pg, cl, seed=20240731, device=cuda_dev, return_clusters=True)
    c2 = atac_binary(lab, cl, pp, seed=20240732)
    # peaks with some variance (an all-zero or all-one column has a zero eigenvalue)
    s2 = c2.sum(0)
    c2 = c2[:, (s2 > 0) & (s2 < n)].contiguous()
    pp = c2.shape[1]
    res = g.fit_multimodal([c1, c2], r, [k, k, k])
    rng = np.random.default_rng(7)
    # sampled Gram entries of the concatenation (FP64 from the counts)
    cols = np.sort(rng.choice(pg + pp, 24, replace=False))
    means = np.concatenate([log1p_col_means(c[i:i + 65536].cpu().numpy() for i in range(0, n, 65536))
                            for c in (c1, c2)])
    cat = torch.cat([c1[:, cols[cols < pg]], c2[:, cols[cols >= pg] - pg]], 1).cpu().numpy().astype(np.float64)
    xc = np.log1p(cat) - means[cols][None, :]
    S = res.S[0].cpu().numpy()
    assert np.max(np.abs(S[np.ix_(cols, cols)] - xc.T @ xc)) <= 2e-5 * np.abs(xc.T @ xc).max()
    # spectra: eigenvalue residuals of the cell axis' lifted vectors and of
    # each feature block; the solve's KKT residual
    E = [e.cpu().numpy() for e in res.E]
    assert np.all(np.diff(E[0]) <= 0) and E[0].shape == (r,)
    for a, blk in ((1, S[:pg, :pg]), (2, S[pg:, pg:])):
        ev = np.linalg.eigvalsh(blk)[::-1]
        np.testing.assert_allclose(E[a], ev, rtol=0, atol=1e-9 * ev[0])
    np.testing.assert_allclose(E[0], np.linalg.eigvalsh(S)[::-1][:r], rtol=1e-9)
    lam = [l.cpu().numpy() for l in res.lam]
    prob = KSProblem(E, [(0, 1), (0, 2)])
    assert rel_kkt(np.concatenate(lam), prob) <= 1e-8
    # networks: cells on sampled rows, features on every row
    rows = np.sort(rng.choice(n, 48, replace=False))
    frac = _sampled_rows_exact(res.V[0].double().cpu().numpy(), lam[0], k, rows, res.idx[0].cpu().numpy()[rows])
    assert frac > 0.5
    assert res.topk_stats[0]["screen_err_ratio"] <= 1.0
    for a, blk in ((1, S[:pg, :pg]), (2, S[pg:, pg:])):
        W = np.linalg.eigh(blk)[1][:, ::-1]
        d = blk.shape[0]
        idx = res.idx[a].cpu().numpy()
        assert idx.shape == (d, k)
        _sampled_rows_exact(W, lam[a], k, np.arange(0, d, max(1, d // 200)), idx[::max(1, d // 200)])
