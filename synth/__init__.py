"""Seeded synthetic inputs for the multi-axis Kronecker-sum GGM fit.

This package only *draws* inputs: planted precision graphs, data matrices and
tensors sampled from a Kronecker-sum normal model, and scRNA-like count
matrices.  It contains none of the fitting method's arithmetic (no Gram, no
eigendecomposition of data, no eigenvalue solve, no reconstruction), so it can
serve both the FP64 oracle and the CUDA path without coupling them.

Recipes (stated once here and in the design notes):

* ``er_precision`` -- Erdos-Renyi graph with mean degree ``deg``
  (edge probability deg/(d-1)), edge weights U[0.1, 0.5] with a random sign,
  diagonal = |row sum| + 1 (strictly diagonally dominant, so positive definite).
* ``ks_normal_matrix`` -- X = V1 (Z / sqrt(l_i + m_j)) V2^T with Z ~ N(0, 1):
  a draw of vec[X] ~ N(0, (Psi2 (+) Psi1)^-1), the Kronecker-sum model of the
  paper's introduction (precision Psi_genes (x) I + I (x) Psi_cells).
* ``ks_normal_tensor`` -- the 3-axis analogue via mode products.
* ``scrna_counts`` -- cells assigned uniformly to clusters; cluster x gene
  log-means offset + N(0, 1); a gene-gene latent z ~ N(0, Psi_g^-1)
  standardised per gene (Psi_g an ER precision); a gamma rate driven by z
  through the Wilson-Hilferty cube transform (shape 1/dispersion, mean m);
  counts ~ Poisson(rate), i.e. negative-binomial-like marginals with
  var ~ m + dispersion * m^2 and a Gaussian-copula-like gene dependence.
* ``atac_binary`` -- Bernoulli accessibility with p ~ Beta(0.5, 10) per
  (cluster, peak), sharing the cell clusters of ``scrna_counts``.
"""

from .graphs import er_precision  # noqa: F401
from .data import (  # noqa: F401
    ks_normal_matrix,
    ks_normal_tensor,
    scrna_counts,
    atac_binary,
    planted_c1,
)
