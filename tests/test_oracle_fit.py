"""Pins of the oracle's multi-modal and tensor fits by reductions to the
two-axis fit (itself pinned in test_oracle_solve / test_oracle_recon)."""

import numpy as np

from oracle.fit import fit_multimodal, fit_tensor, fit_two_axis
from oracle.gram import log1p_centre
from oracle.solve import default_eps
from synth import scrna_counts


def _x(n, p, seed):
    return log1p_centre(scrna_counts(n, p, 4, seed=seed).numpy())


def test_one_modality_is_the_two_axis_fit():
    x = _x(300, 40, 3)
    mm = fit_multimodal([x], 8, [5, 4])
    ta = fit_two_axis(x, 8, 40, 5, 4)
    np.testing.assert_allclose(mm.E[0], ta.e_rows, rtol=1e-12)
    np.testing.assert_allclose(mm.E[1], ta.e_cols, rtol=1e-12)
    np.testing.assert_allclose(mm.lam[0][:, None] + mm.lam[1][None, :], ta.lam_rows[:, None] + ta.lam_cols[None, :],
                               rtol=1e-10)
    assert np.array_equal(mm.topk[0][0], ta.topk_rows[0])
    assert np.array_equal(mm.topk[1][0], ta.topk_cols[0])


def test_duplicated_modality_halves_into_the_two_axis_fit():
    # [X X]: the concatenation's column Gram has the cell spectrum doubled;
    # f(lam, mu, nu) with nu = mu is twice the two-axis f with the original
    # cell spectrum, so the fit is the two-axis fit (same eps), and the lift
    # through [X X] returns the same cell vectors
    x = _x(250, 30, 5)
    e2 = fit_two_axis(x, 6, 30, 4, 3)
    eps = default_eps([e2.e_rows, e2.e_cols], [(0, 1)])
    ta = fit_two_axis(x, 6, 30, 4, 3, eps=eps)
    mm = fit_multimodal([x, x], 6, [4, 3, 3], eps=[eps[0]] * 3)
    np.testing.assert_allclose(mm.E[0], 2 * ta.e_rows, rtol=1e-12)
    np.testing.assert_allclose(mm.E[1], ta.e_cols, rtol=1e-12)
    np.testing.assert_allclose(mm.E[2], ta.e_cols, rtol=1e-12)
    np.testing.assert_allclose(mm.lam[1], mm.lam[2], rtol=1e-9)
    np.testing.assert_allclose(mm.lam[0][:, None] + mm.lam[1][None, :], ta.lam_rows[:, None] + ta.lam_cols[None, :],
                               rtol=1e-9)
    psi_mm = (mm.V[0] * mm.lam[0]) @ mm.V[0].T
    psi_ta = (ta.v_rows * ta.lam_rows) @ ta.v_rows.T
    np.testing.assert_allclose(psi_mm, psi_ta, atol=1e-9 * np.abs(psi_ta).max())


def test_tensor_with_a_unit_axis_is_the_matrix_fit():
    # T = X[:, :, None]: the third axis' Gram is the 1 x 1 ||X||^2 = tr E_0,
    # so E_2 nu = E_0 . (nu 1) and the third axis folds into the first: the
    # sums lam_i + mu_j + nu equal the two-axis fit's lam_i + mu_j, and the
    # networks of the first two axes are the matrix fit's
    x = np.random.default_rng(9).standard_normal((5, 5))  # full rank on both axes
    tf = fit_tensor(x[:, :, None], [2, 2, None])
    ta = fit_two_axis(x, 5, 5, 2, 2)
    assert tf.E[2].shape == (1,) and tf.topk[2] is None
    np.testing.assert_allclose(tf.E[2][0], np.sum(x * x), rtol=1e-12)
    s3 = tf.lam[0][:, None] + tf.lam[1][None, :] + tf.lam[2][0]
    s2 = ta.lam_rows[:, None] + ta.lam_cols[None, :]
    np.testing.assert_allclose(s3, s2, rtol=1e-8)
    assert np.array_equal(tf.topk[1][0], ta.topk_cols[0])
