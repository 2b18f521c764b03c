"""GPU parity of the global top-n edges (the global threshold of Algorithm
1's last loop) derived from per-row top-k lists, against the oracle's
derivation from the same lists (bit-exact pairs and values, the same
certificate) and, where certified, against the oracle's global top-n of the
network itself."""

import numpy as np
import pytest
import torch

from oracle import recon as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g(cuda_dev):
    import paper_2407_19892_gb300 as pkg
    pkg.load()
    return pkg


def _gpu_topn(g, dev, idx, val, n):
    i, j, v, cert = g.topn_edges(torch.from_numpy(np.ascontiguousarray(idx, dtype=np.int32)).to(dev),
                                 torch.from_numpy(np.ascontiguousarray(val, dtype=np.float32)).to(dev), n)
    return i.cpu().numpy(), j.cpu().numpy(), v.cpu().numpy(), cert


def _same_as_oracle_derivation(g, dev, idx, val, n):
    gi, gj, gv, gc = _gpu_topn(g, dev, idx, val, n)
    oi, oj, ov, oc = orc.topn_from_row_lists(idx, val.astype(np.float32).astype(np.float64), n)
    assert np.array_equal(gi, oi) and np.array_equal(gj, oj)
    assert np.array_equal(gv, ov.astype(np.float32))
    assert gc == oc
    return gi, gj, gv, gc


@pytest.mark.parametrize("d,r,k,n", [(3000, 8, 10, 500), (257, 5, 6, 40), (1500, 20, 16, 3000)])
def test_from_gpu_lists_matches_the_oracle(g, cuda_dev, d, r, k, n):
    rng = np.random.default_rng(d + r)
    V = rng.standard_normal((d, r))
    lam = rng.uniform(0.2, 2.0, r)
    idx, val, _ = g.topk_network(torch.from_numpy(V.astype(np.float32)).to(cuda_dev),
                                 torch.from_numpy(lam).to(cuda_dev), k)
    idx, val = idx.cpu().numpy(), val.cpu().numpy()
    gi, gj, gv, cert = _same_as_oracle_derivation(g, cuda_dev, idx, val, n)
    if cert:
        # the network's own global top-n (FP64, from the same FP32 V)
        ti, tj, tv = orc.topn_edges(V.astype(np.float32).astype(np.float64), lam, n + 1)
        mag = np.abs(tv)
        if mag[n - 1] - mag[n] > 1e-5 * mag[n - 1]:
            assert set(zip(gi.tolist(), gj.tolist())) == set(zip(ti[:n].tolist(), tj[:n].tolist()))


def test_ties_are_ordered_by_pair(g, cuda_dev):
    # duplicated rows: equal magnitudes in many pairs
    rng = np.random.default_rng(3)
    V = np.repeat(rng.standard_normal((40, 3)), 4, axis=0)
    lam = rng.uniform(0.5, 1.5, 3)
    idx, val = orc.topk_rows(V, lam, 7)
    _same_as_oracle_derivation(g, cuda_dev, idx, val.astype(np.float32), 100)


def test_clique_is_not_certified_with_short_lists(g, cuda_dev):
    rng = np.random.default_rng(14)
    d = 40
    M = 10.0 * np.eye(d) + 0.01 * rng.standard_normal((d, d))
    M[:12, :12] += 5.0 + 0.1 * rng.standard_normal((12, 12))
    M = 0.5 * (M + M.T)
    lam, V = np.linalg.eigh(M)
    for k, want in ((5, False), (11, False), (12, True)):
        idx, val = orc.topk_rows(V, lam, k)
        *_, cert = _same_as_oracle_derivation(g, cuda_dev, idx, val.astype(np.float32), 66)
        assert cert == want


def test_fewer_pairs_than_asked(g, cuda_dev):
    rng = np.random.default_rng(5)
    V = rng.standard_normal((30, 4))
    idx, val = orc.topk_rows(V, rng.uniform(0.5, 1.0, 4), 2)
    gi, gj, gv, cert = _gpu_topn(g, cuda_dev, idx, val.astype(np.float32), 60)
    assert len(gi) < 60 and not cert
    _same_as_oracle_derivation(g, cuda_dev, idx, val.astype(np.float32), 60)


def test_one_million_rows_of_lists(g, cuda_dev):
    # lists at the 1M-cell workload's size (k = 10): distinct off-diagonal
    # columns per row, values on a 1/64 grid (many equal magnitudes), each
    # row sorted by magnitude like a top-k list; pairs listed from both ends
    # occur where offsets coincide
    rng = np.random.default_rng(6)
    d, k, n = 1_000_000, 10, 200_000
    off = np.cumsum(rng.integers(1, 40, size=(d, k)), axis=1)
    idx = (np.arange(d)[:, None] + off) % d
    val = np.round(rng.standard_normal((d, k)) * 64.0) / 64.0
    val = np.take_along_axis(val, np.argsort(-np.abs(val), axis=1, kind="stable"), 1)
    _same_as_oracle_derivation(g, cuda_dev, idx, val.astype(np.float32), n)
