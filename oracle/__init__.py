"""FP64 CPU oracle for the improved multi-axis GmGM fit (arXiv 2407.19892).

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain, obviously-correct
statement of what the GPU path computes.  Only the test suite, the smoke check
and the benchmark's CPU-baseline leg may import it; the product path
(``paper_2407_19892_gb300``) never does, and this package never imports the
product path.  The two share no code: the only common dependency is the
``synth`` input generators, which hold none of the method's arithmetic.

Each function cites the part of the paper it follows:

* ``gram``      -- sufficient statistics S_l = mat_l[D] mat_l[D]^T
                   (Section "Algorithm", the concatenated-matricisation identity;
                   Algorithm 1, first loop).
* ``spectra``   -- top-r eigenpairs of S_l and the dual lift of the large axis
                   (Theorem 1; Algorithm 1, singular vectors / squared values).
* ``solve``     -- the eigenvalue problem: minimise
                   sum_l E_l . Lam_l - sum_gamma sum_grid log(sum_l lam_l,idx)
                   over the box Lam_l >= eps_l (Proposition on the eigenvalue
                   gradient; the elementwise form in the existence lemma;
                   Algorithm 1's gradient step), by a projected Newton method,
                   plus the paper's literal gradient iteration.
* ``recon``     -- Psi_l = V_l diag(Lam_l) V_l^T, its per-row top-k and the
                   global top-n edges (Algorithm 1, last loop: threshold with
                   recomposition; the complexity appendix's heap of size n_l).
* ``kron``      -- Kronecker sums and the dense (brute-force) likelihood used to
                   pin the rest on tiny problems (Introduction's Kronecker-sum
                   definition; the model equation; appendix on the singular
                   distribution).
* ``mlp``       -- FP64 forward/backward of the warm-start network.
* ``sparse``    -- the column Gram and the dual lift of log1p(counts) with
                   centring, from the sparse matrix and rank-one corrections
                   (the appendix on preserving input sparsity).
* ``skeptic``   -- rank-based statistics: per-row minimum ranks, normal
                   scores Phi^-1(rank / (n + 1)) and their Gram (Section "The
                   model", the Nonparanormal Skeptic; Section "Algorithm",
                   the COCA form; the worked example of the appendix on
                   preserving input sparsity).

Pins live in ``tests/test_oracle_*.py`` (``-m "not gpu"``).
"""
