"""The two-axis fit with its cells split over processes (one per GPU).

Section "Algorithm": the gene Gram S = X^T X is a sum over blocks of cells,
so each process holds a block of rows (cells) of the count matrix and the
fit needs five exchanges, all of them small except the last:

  1. column sums of log1p(counts) (p FP64) and the cell counts: all-reduce;
  2. the Gram partials X_b^T X_b (p x p FP64, 32 MB at 2,000 genes):
     all-reduce;
  3. the gene spectrum E (p FP64) and the top-r eigenvectors W_r (p x r
     FP64) from rank 0: broadcast (the eigendecomposition runs once);
  4. the eigenvalues Lam of the solve on rank 0 (r + p FP64): broadcast;
  5. the cell vectors U_b (n_b x r FP32, 200 MB in all at 1M cells x 50):
     all-gather, after which every process computes the top-k lists of the
     rows it owns against all cells (no list is exchanged).

The dual lift is local (U_b = X_b W_r diag(E_r)^-1/2).  The gene network
depends only on S and Lam and is computed by rank 0.  Which arithmetic runs
on a process is a backend's business (``GpuBackend``: this library's
kernels); the exchanges are the communicator's (``TorchComm``:
``torch.distributed``, with tensors staged through host memory when the
process group is gloo).
"""

from dataclasses import dataclass

import torch

from . import _lib as L
from . import api


class TorchComm:
    """Collectives over the default torch.distributed process group.  With
    a gloo group, CUDA tensors are copied to host memory for the exchange
    and back.  ``log`` records (operation, shape, dtype) of every exchange."""

    def __init__(self):
        import torch.distributed as dist
        self.dist = dist
        self.active = dist.is_available() and dist.is_initialized()
        self.rank = dist.get_rank() if self.active else 0
        self.world = dist.get_world_size() if self.active else 1
        self.host_staging = self.active and dist.get_backend() == "gloo"
        self.log = []

    def _stage(self, t):
        return t.cpu() if (self.host_staging and t.is_cuda) else t

    def all_reduce_sum(self, t):
        self.log.append(("all_reduce", tuple(t.shape), str(t.dtype)))
        if self.world == 1:
            return t
        s = self._stage(t)
        self.dist.all_reduce(s)
        if s is not t:
            t.copy_(s)
        return t

    def broadcast(self, t, src=0):
        self.log.append(("broadcast", tuple(t.shape), str(t.dtype)))
        if self.world == 1:
            return t
        s = self._stage(t)
        self.dist.broadcast(s, src)
        if s is not t:
            t.copy_(s)
        return t

    def all_gather_rows(self, t):
        """Concatenate every rank's t along dim 0 (row counts may differ)."""
        self.log.append(("all_gather", tuple(t.shape), str(t.dtype)))
        if self.world == 1:
            return t
        s = self._stage(t)
        n = torch.tensor([s.shape[0]], dtype=torch.int64, device=s.device)
        ns = [torch.zeros_like(n) for _ in range(self.world)]
        self.dist.all_gather(ns, n)
        ns = [int(x.item()) for x in ns]
        pad = torch.zeros((max(ns),) + tuple(s.shape[1:]), dtype=s.dtype, device=s.device)
        pad[:s.shape[0]] = s
        parts = [torch.empty_like(pad) for _ in range(self.world)]
        self.dist.all_gather(parts, pad)
        out = torch.cat([q[:m] for q, m in zip(parts, ns)], dim=0)
        return out.to(t.device)


class GpuBackend:
    """The fit's arithmetic on this process' GPU, through the library."""

    def __init__(self, gram_prec=L.BF16X3, topk_prec=L.BF16, tol=1e-9, h=None):
        self.gram_prec, self.topk_prec, self.tol, self.h = gram_prec, topk_prec, tol, h

    def colsum(self, counts):
        h = self.h or api.handle(counts.device)
        n, p = counts.shape
        cs = torch.empty(p, dtype=torch.float64, device=counts.device)
        h.check(h.lib.gmgm_colsum_log1p(h.h, n, p, api._ptr(counts), counts.stride(0), api._ptr(cs), 0))
        return cs

    def centre(self, counts, colsum, n_total):
        h = self.h or api.handle(counts.device)
        n, p = counts.shape
        x = torch.empty_like(counts)
        split = self.gram_prec != L.FP32
        ld_t = ((n + 63) // 64) * 64 if split else 0
        hi = torch.empty(p, ld_t, dtype=torch.bfloat16, device=counts.device) if split else None
        lo = torch.empty(p, ld_t, dtype=torch.bfloat16, device=counts.device) if split else None
        h.check(h.lib.gmgm_centre(h.h, n, p, api._ptr(counts), counts.stride(0), api._ptr(colsum), n_total,
                                  api._ptr(x), x.stride(0), api._ptr(hi), api._ptr(lo), ld_t))
        return x, hi, lo, ld_t

    def gram(self, x, hi, lo, ld_t):
        return api.gram(x, L.SIDE_COLS, self.gram_prec, xt_hi=hi, xt_lo=lo, ld_t=ld_t, h=self.h)

    def spectra(self, S, r):
        return api.spectra(S, S.shape[0], rv=r, h=self.h)

    def lift(self, x, hi, lo, ld_t, W, E):
        return api.lift(x, W, E, W.shape[1], xt_hi=hi, xt_lo=lo, ld_t=ld_t, h=self.h)

    def eigsolve(self, e_rows, e_cols):
        (lr, lc), st = api.eigsolve([e_rows, e_cols], [(0, 1)], tol=self.tol, h=self.h)
        return lr, lc, st

    def topk_rows(self, U, lam, k, row0, m):
        idx, val, _ = api.topk_network_rows(U, lam, k, row0, m, self.topk_prec, h=self.h)
        return idx, val

    def topk_gram(self, S, lam, k):
        idx, val, _ = api.topk_network_gram(S, lam, k, L.FP32, h=self.h)
        return idx, val


@dataclass
class ShardedResult:
    row0: int            # this process' first cell
    n_total: int         # cells over all processes
    e_cols: torch.Tensor  # the gene spectrum (all p values, descending)
    lam_rows: torch.Tensor
    lam_cols: torch.Tensor
    idx_rows: torch.Tensor  # top-k lists of this process' cells (n_local x k_rows)
    val_rows: torch.Tensor
    idx_cols: torch.Tensor  # gene network (rank 0), else None
    val_cols: torch.Tensor
    solve: dict


def fit_two_axis_sharded(counts, r_rows: int, k_rows: int, k_cols: int, backend=None, comm=None) -> ShardedResult:
    """Algorithm 1 on a count matrix whose cells (rows) are split over the
    processes of ``comm``: this process passes its block of rows (n_b x p
    FP32 counts); blocks are ordered by rank.  Preprocessing (log1p, then
    centring by the global column means), the gene Gram, its spectrum, the
    dual lift, the eigenvalue solve and both networks, with the exchanges
    listed in the module docstring.  The gene axis is at full rank."""
    backend = backend or GpuBackend()
    comm = comm or TorchComm()
    n_local, p = counts.shape
    # 1. global column means
    cs = backend.colsum(counts)
    nn = torch.tensor([float(n_local)], dtype=torch.float64, device=cs.device)
    comm.all_reduce_sum(cs)
    comm.all_reduce_sum(nn)
    n_total = int(round(float(nn.item())))
    x, hi, lo, ld_t = backend.centre(counts, cs, n_total)
    # 2. the gene Gram, summed over the blocks of cells
    S = backend.gram(x, hi, lo, ld_t)
    comm.all_reduce_sum(S)
    # 3. spectrum on rank 0
    E = torch.empty(p, dtype=torch.float64, device=S.device)
    W = torch.empty(p, r_rows, dtype=torch.float64, device=S.device)
    if comm.rank == 0:
        e0, w0 = backend.spectra(S, r_rows)
        E.copy_(e0)
        W.copy_(w0)
    comm.broadcast(E)
    comm.broadcast(W)
    e_rows = E[:r_rows].contiguous()
    U = backend.lift(x, hi, lo, ld_t, W, e_rows)
    # 4. the solve on rank 0
    lam = torch.empty(r_rows + p, dtype=torch.float64, device=S.device)
    st = {}
    if comm.rank == 0:
        lr, lc, st = backend.eigsolve(e_rows, E)
        lam[:r_rows].copy_(lr)
        lam[r_rows:].copy_(lc)
    comm.broadcast(lam)
    lam_rows, lam_cols = lam[:r_rows].contiguous(), lam[r_rows:].contiguous()
    # 5. all cells' vectors; this process' rows of the cell network
    sizes = torch.zeros(comm.world, dtype=torch.float64, device=S.device)
    sizes[comm.rank] = float(n_local)
    comm.all_reduce_sum(sizes)
    row0 = int(round(float(sizes[:comm.rank].sum().item())))
    U_all = comm.all_gather_rows(U)
    idx_r, val_r = backend.topk_rows(U_all, lam_rows, k_rows, row0, n_local)
    idx_c = val_c = None
    if comm.rank == 0:
        idx_c, val_c = backend.topk_gram(S, lam_cols, k_cols)
    return ShardedResult(row0, n_total, E, lam_rows, lam_cols, idx_r, val_r, idx_c, val_c, st)
