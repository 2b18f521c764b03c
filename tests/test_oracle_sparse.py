"""Pins of the sparse-input oracle (oracle/sparse.py): the rank-one forms
equal the dense computation they replace."""

import numpy as np
import scipy.sparse as sp

from oracle import gram as og
from oracle import sparse as osp_
from oracle import spectra as ospec
from synth import scrna_counts


def _counts():
    c = scrna_counts(600, 45, 4, seed=9).numpy().astype(np.float64)
    assert (c == 0).mean() > 0.3  # a sparse workload
    return c


def test_log1p_keeps_the_sparsity_pattern():
    c = _counts()
    x = osp_.log1p_sparse(sp.csr_matrix(c))
    assert x.nnz == np.count_nonzero(c)
    np.testing.assert_array_equal(x.toarray(), np.log1p(c))


def test_centred_gram_equals_the_dense_gram_of_centred_data():
    c = _counts()
    g, mu = osp_.centred_gram_sparse(osp_.log1p_sparse(sp.csr_matrix(c)))
    xc = og.log1p_centre(c)
    ref = og.gram(xc, 1)
    assert np.max(np.abs(g - ref)) <= 1e-9 * np.abs(ref).max()
    np.testing.assert_allclose(mu, np.log1p(c).mean(axis=0), rtol=1e-13)


def test_centred_lift_equals_the_dense_lift():
    c = _counts()
    x = osp_.log1p_sparse(sp.csr_matrix(c))
    g, mu = osp_.centred_gram_sparse(x)
    e, w = ospec.top_eigh(g, 7)
    got = osp_.centred_lift_sparse(x, mu, w, e)
    ref = ospec.dual_lift(og.log1p_centre(c), w, e)
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.abs(ref).max()
    # the lifted vectors are orthonormal (they are X_c's left singular vectors)
    assert np.max(np.abs(got.T @ got - np.eye(7))) <= 1e-8
