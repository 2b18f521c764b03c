"""Seeded synthetic data: Kronecker-sum normal draws and scRNA/ATAC-like counts."""

import math

import numpy as np
import torch

from .graphs import er_precision


def _eig_sample_scales(psi: np.ndarray):
    """Eigenpairs of a planted precision (sampling only, not the fitted method)."""
    w, v = np.linalg.eigh(psi)
    return w, v


def ks_normal_matrix(psi_rows: np.ndarray, psi_cols: np.ndarray,
                     rng: np.random.Generator) -> np.ndarray:
    """One draw X (d1 x d2) with precision Psi_cols (x) I + I (x) Psi_rows.

    X = V1 (Z / sqrt(l_i + m_j)) V2^T, Z ~ N(0, 1), where (l, V1) and (m, V2)
    are the eigenpairs of the row-axis and column-axis precisions.  Then
    -1/2 vec[X]^T (Psi2 (+) Psi1) vec[X] = -1/2 sum_ij (l_i + m_j) Z'_ij^2.
    """
    l, v1 = _eig_sample_scales(psi_rows)
    m, v2 = _eig_sample_scales(psi_cols)
    z = rng.standard_normal((len(l), len(m)))
    y = z / np.sqrt(l[:, None] + m[None, :])
    return v1 @ y @ v2.T


def ks_normal_tensor(psis, rng: np.random.Generator) -> np.ndarray:
    """One draw of a 3-axis tensor with Kronecker-sum precision over its axes."""
    pairs = [_eig_sample_scales(p) for p in psis]
    ls = [w for w, _ in pairs]
    s = ls[0][:, None, None] + ls[1][None, :, None] + ls[2][None, None, :]
    y = rng.standard_normal(s.shape) / np.sqrt(s)
    v1, v2, v3 = (v for _, v in pairs)
    return np.einsum("abc,xa,yb,zc->xyz", y, v1, v2, v3, optimize=True)


def planted_c1(seed: int = 20240728, d1: int = 200, d2: int = 100, deg: float = 4.0):
    """The small plain-FP64 case: planted ER precisions, one KS-normal draw.

    Returns (X, Psi_rows, Psi_cols) as float64 numpy arrays.
    """
    rng = np.random.Generator(np.random.Philox(seed))
    psi1 = er_precision(d1, deg, rng)
    psi2 = er_precision(d2, deg, rng)
    x = ks_normal_matrix(psi1, psi2, rng)
    return x, psi1, psi2


def scrna_counts(n_cells: int, n_genes: int, n_clusters: int, seed: int,
                 device="cpu", deg: float = 5.0, dispersion: float = 0.5,
                 offset: float = -1.0, chunk: int = 1 << 17,
                 out: torch.Tensor = None, return_clusters: bool = False):
    """scRNA-like count matrix (n_cells x n_genes, float32, row-major).

    Cells are assigned uniformly to ``n_clusters`` clusters; cluster x gene
    means are exp(offset + N(0, 1)); a gene-gene latent z ~ N(0, Psi_g^-1)
    (Psi_g an ER precision of mean degree ``deg``) is standardised per gene
    and drives a gamma rate through the Wilson-Hilferty transform
    rate = m * (1 - 1/(9k) + z / (3 sqrt(k)))^3, k = 1/dispersion; counts are
    Poisson(rate).  Generated in row chunks on ``device``.
    """
    dev = torch.device(device)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    rng = np.random.Generator(np.random.Philox(seed))
    psi_g = er_precision(n_genes, deg, rng)
    chol = np.linalg.cholesky(psi_g)
    linv = np.linalg.inv(chol)  # z_i^T = y_i^T L^-1 has covariance Psi_g^-1
    std = np.sqrt((linv * linv).sum(axis=0))
    mix = torch.from_numpy(linv / std[None, :]).to(dev, torch.float32)
    logm = offset + torch.randn(n_clusters, n_genes, generator=g, device=dev)
    means = torch.exp(logm)
    cl = torch.randint(0, n_clusters, (n_cells,), generator=g, device=dev)
    if out is None:
        out = torch.empty(n_cells, n_genes, dtype=torch.float32, device=dev)
    k = 1.0 / dispersion
    a = 1.0 - 1.0 / (9.0 * k)
    b = 1.0 / (3.0 * math.sqrt(k))
    for r0 in range(0, n_cells, chunk):
        r1 = min(n_cells, r0 + chunk)
        y = torch.randn(r1 - r0, n_genes, generator=g, device=dev)
        z = y @ mix
        wh = torch.clamp(a + b * z, min=0.0) ** 3
        rate = means[cl[r0:r1]] * wh
        out[r0:r1] = torch.poisson(rate, generator=g)
        del y, z, wh, rate
    if return_clusters:
        return out, cl, psi_g
    return out


def atac_binary(clusters: torch.Tensor, n_clusters: int, n_peaks: int, seed: int,
                a: float = 0.5, b: float = 10.0, chunk: int = 1 << 17,
                out: torch.Tensor = None):
    """Binary accessibility (n_cells x n_peaks, float32): Bernoulli with
    p ~ Beta(a, b) per (cluster, peak), sharing the cells' cluster labels."""
    dev = clusters.device
    rng = np.random.Generator(np.random.Philox(seed))
    p = torch.from_numpy(rng.beta(a, b, size=(n_clusters, n_peaks))).to(dev, torch.float32)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    n = clusters.numel()
    if out is None:
        out = torch.empty(n, n_peaks, dtype=torch.float32, device=dev)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        out[r0:r1] = torch.bernoulli(p[clusters[r0:r1]], generator=g)
    return out
