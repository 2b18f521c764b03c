"""GPU parity of the sparse-input path (the appendix "Preserving input
sparsity"): a CSR count matrix preprocessed straight into the BF16 planes of
X^T (sparse log1p part plus the rank-one centring term), against the dense
preprocessing of the same counts and the oracle's sparse forms, and the
whole two-axis fit from the planes against the oracle's fit."""

import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import sparse as osp_
from oracle.fit import fit_two_axis as ofit
from oracle.gram import log1p_centre
from synth import scrna_counts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g(cuda_dev):
    import paper_2407_19892_gb300 as pkg
    pkg.load()
    return pkg


def _csr(counts, dev):
    c = sp.csr_matrix(counts)
    c.sort_indices()
    return (torch.from_numpy(c.indptr.astype(np.int64)).to(dev), torch.from_numpy(c.indices.astype(np.int32)).to(dev),
            torch.from_numpy(c.data.astype(np.float32)).to(dev), c)


@pytest.mark.parametrize("n,p", [(5000, 300), (1001, 77), (64, 2000), (3, 5)])
def test_planes_from_csr_match_the_dense_path_and_the_oracle(g, cuda_dev, n, p):
    counts = scrna_counts(n, p, 6, seed=700 + n).numpy()
    counts[n // 2] = 0.0  # an empty row
    ip, ix, dv, c = _csr(counts, cuda_dev)
    hi, lo, ld_t, mu = g.preprocess_csr(ip, ix, dv, n, p)
    assert g.handle(cuda_dev).device_status() == 0
    x64 = log1p_centre(counts)
    np.testing.assert_allclose(mu.cpu().numpy(), np.log1p(counts.astype(np.float64)).mean(0), rtol=2e-7, atol=1e-12)
    xt = (hi.float() + lo.float()).cpu().numpy()
    assert np.all(xt[:, n:] == 0)
    scale = max(1.0, np.abs(x64).max())
    assert np.max(np.abs(xt[:, :n] - x64.T)) <= 2 ** -16 * scale
    # the dense path's planes of the same counts
    _, dhi, dlo, dld = g.preprocess(torch.from_numpy(counts).to(cuda_dev), split=True)
    assert dld == ld_t
    dxt = (dhi.float() + dlo.float()).cpu().numpy()
    assert np.max(np.abs(xt - dxt)) <= 2 ** -16 * scale
    if n >= 64:
        # the Gram from the planes = the oracle's sparse part + rank-one term
        S = g.gram(None, g.SIDE_COLS, g.BF16X3, xt_hi=hi, xt_lo=lo, ld_t=ld_t, rows=n, cols=p).cpu().numpy()
        ref, mu_ref = osp_.centred_gram_sparse(osp_.log1p_sparse(c))
        assert np.max(np.abs(S - ref)) <= 2e-5 * np.abs(ref).max()


def test_fit_from_csr_matches_the_oracle(g, cuda_dev):
    n, p, r, k = 20_000, 400, 20, 10
    counts = scrna_counts(n, p, 8, seed=777).numpy()
    ip, ix, dv, _ = _csr(counts, cuda_dev)
    hi, lo, ld_t, _ = g.preprocess_csr(ip, ix, dv, n, p)
    res = g.fit_two_axis(None, r, p, k, k, gram_prec=g.BF16X3, topk_prec=g.BF16, xt_hi=hi, xt_lo=lo, ld_t=ld_t,
                         rows=n)
    ref = ofit(log1p_centre(counts), r, p, k, k)
    sg = res.lam_rows.cpu().numpy()[:, None] + res.lam_cols.cpu().numpy()[None, :]
    sr = ref.lam_rows[:, None] + ref.lam_cols[None, :]
    assert np.max(np.abs(sg - sr) / sr) <= 1e-4
    assert res.v_rows.shape == (n, r)
    # the dense path on the same counts gives the same fit to its rounding
    x, dhi, dlo, dld = g.preprocess(torch.from_numpy(counts).to(cuda_dev), split=True)
    dres = g.fit_two_axis(x, r, p, k, k, gram_prec=g.BF16X3, topk_prec=g.BF16, xt_hi=dhi, xt_lo=dlo, ld_t=dld)
    sd = dres.lam_rows.cpu().numpy()[:, None] + dres.lam_cols.cpu().numpy()[None, :]
    assert np.max(np.abs(sg - sd) / sd) <= 1e-5


@pytest.mark.parametrize("case", ["unsorted", "negative", "out_of_range"])
def test_invalid_csr_entries_set_the_status_bit(g, cuda_dev, case):
    counts = np.ones((10, 6), dtype=np.float32)
    ip, ix, dv, _ = _csr(counts, cuda_dev)
    ix, dv = ix.clone(), dv.clone()
    if case == "unsorted":
        ix[2], ix[3] = int(ix[3]), int(ix[2])
    elif case == "negative":
        dv[5] = -2.0
    else:
        ix[7] = 6
    g.preprocess_csr(ip, ix, dv, 10, 6)
    assert g.handle(cuda_dev).device_status() == 0x20
