"""Parity of the multi-modal and 3-axis fits with the FP64 oracle.

Modalities sharing the cell axis (scRNA-like counts + ATAC-like binary
accessibility of the same cells) and a 3-axis tensor with planted
Kronecker-sum precision.  Judged as the two-axis fit is: spectra and the
eigenvalue sums against the oracle's own fit (1e-4 relative), and every
network stage-wise (the oracle's FP64 top-k of the GPU's own vectors and
eigenvalues, bit-exact where the k-th/(k+1)-th gap exceeds 1e-5)."""

import numpy as np
import pytest
import torch

import oracle.recon as orc
from oracle.fit import fit_multimodal as ofit_mm, fit_tensor as ofit_t
from oracle.gram import log1p_centre
from synth import atac_binary, er_precision, ks_normal_tensor, scrna_counts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_2407_19892_gb300 as g
    g.load()
    return g


def _check_net(V64, lam, k, idx, val):
    ref_i, ref_v = orc.topk_rows(V64, lam, k)
    gap = orc.topk_gap(V64, lam, k)
    ok = gap > 1e-5
    assert np.array_equal(np.sort(idx[ok], 1), np.sort(ref_i[ok], 1))
    np.testing.assert_allclose(np.take_along_axis(val, np.argsort(idx, 1), 1)[ok],
                               np.take_along_axis(ref_v, np.argsort(ref_i, 1), 1)[ok].astype(np.float32),
                               rtol=1e-6, atol=1e-30)
    return ok.mean()


def _sums_close(la, lb, ra, rb, tol=1e-4):
    sa = la[:, None] + lb[None, :]
    sr = ra[:, None] + rb[None, :]
    return float(np.max(np.abs(sa - sr) / sr)) <= tol


def test_fit_multimodal_rna_plus_atac(g, cuda_dev):
    n, p_rna, p_atac, clusters = 3000, 120, 200, 6
    c1, cl, _ = scrna_counts(n, p_rna, clusters, seed=41, return_clusters=True)
    c2 = atac_binary(cl, clusters, p_atac, seed=42)
    c2 = c2[:, (c2.sum(0) > 0) & (c2.sum(0) < n)].contiguous()  # peaks with some variance
    res = g.fit_multimodal([c1.to(cuda_dev), c2.to(cuda_dev)], 20, [10, 8, 8])
    ref = ofit_mm([log1p_centre(c1.numpy()), log1p_centre(c2.numpy())], 20, [10, 8, 8])
    E = [e.cpu().numpy() for e in res.E]
    lam = [l.cpu().numpy() for l in res.lam]
    for a in range(3):
        np.testing.assert_allclose(E[a], ref.E[a], rtol=0, atol=1e-4 * ref.E[a][0])
    assert res.solve["status"] == 0
    assert _sums_close(lam[0], lam[1], ref.lam[0], ref.lam[1])
    assert _sums_close(lam[0], lam[2], ref.lam[0], ref.lam[2])
    # feature axes: their networks come from the Gram blocks; the stage-wise
    # check uses FP64 eigenvectors of the GPU's own blocks
    Vs = [res.V[0].double().cpu().numpy()] + [np.linalg.eigh(res.S[a].cpu().numpy())[1][:, ::-1] for a in (1, 2)]
    fracs = [_check_net(Vs[a], lam[a], [10, 8, 8][a], res.idx[a].cpu().numpy(), res.val[a].cpu().numpy())
             for a in range(3)]
    assert fracs[0] > 0.5


def test_fit_tensor_planted_three_axis(g, cuda_dev):
    # the 3-axis case at its full size: 50 x 400 x 300, planted ER precisions
    rng = np.random.default_rng(20240730)
    psis = [er_precision(d, 4.0, rng) for d in (50, 400, 300)]
    t = ks_normal_tensor(psis, rng)
    res = g.fit_tensor(torch.from_numpy(t.astype(np.float32)).to(cuda_dev), [5, 5, 5])
    ref = ofit_t(t.astype(np.float32).astype(np.float64), [5, 5, 5])
    E = [e.cpu().numpy() for e in res.E]
    lam = [l.cpu().numpy() for l in res.lam]
    for a in range(3):
        np.testing.assert_allclose(E[a], ref.E[a], rtol=0, atol=1e-6 * ref.E[a][0])
    s = lam[0][:, None, None] + lam[1][None, :, None] + lam[2][None, None, :]
    sr = ref.lam[0][:, None, None] + ref.lam[1][None, :, None] + ref.lam[2][None, None, :]
    assert float(np.max(np.abs(s - sr) / sr)) <= 1e-4
    for a in range(3):
        W = np.linalg.eigh(res.S[a].cpu().numpy())[1][:, ::-1]
        frac = _check_net(W, lam[a], 5, res.idx[a].cpu().numpy(), res.val[a].cpu().numpy())
        assert frac > 0.5
