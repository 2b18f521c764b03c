"""Test double for the cell-sharded fit: the per-process arithmetic of
``paper_2407_19892_gb300.sharded`` done by the FP64 oracle on CPU tensors,
so the exchange logic runs on gloo ranks without a GPU."""

import numpy as np
import torch

from oracle.gram import gram
from oracle.recon import topk_rows
from oracle.solve import solve_newton, two_axis_problem
from oracle.spectra import dual_lift, top_eigh


def _np(t):
    return t.detach().cpu().numpy()


class OracleBackend:
    def colsum(self, counts):
        return torch.from_numpy(np.log1p(_np(counts).astype(np.float64)).sum(axis=0))

    def centre(self, counts, colsum, n_total):
        x = np.log1p(_np(counts).astype(np.float64)) - (_np(colsum) / n_total)[None, :]
        return torch.from_numpy(x), None, None, 0

    def gram(self, x, hi, lo, ld_t):
        return torch.from_numpy(gram(_np(x), 1))

    def spectra(self, S, r):
        e, w = top_eigh(_np(S), S.shape[0])
        return torch.from_numpy(e.copy()), torch.from_numpy(np.ascontiguousarray(w[:, :r]))

    def lift(self, x, hi, lo, ld_t, W, E):
        return torch.from_numpy(dual_lift(_np(x), _np(W), _np(E)))

    def eigsolve(self, e_rows, e_cols):
        prob = two_axis_problem(_np(e_rows), _np(e_cols))
        lam, info = solve_newton(prob)
        r = len(e_rows)
        return torch.from_numpy(lam[:r].copy()), torch.from_numpy(lam[r:].copy()), {"converged": info.converged}

    def topk_rows(self, U, lam, k, row0, m):
        idx, val = topk_rows(_np(U), _np(lam), k, rows=np.arange(row0, row0 + m))
        return torch.from_numpy(idx), torch.from_numpy(val)

    def topk_gram(self, S, lam, k):
        _, w = top_eigh(_np(S), S.shape[0])
        idx, val = topk_rows(w, _np(lam), k)
        return torch.from_numpy(idx), torch.from_numpy(val)
