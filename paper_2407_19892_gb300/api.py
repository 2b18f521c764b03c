"""Python surface over the C ABI: torch device tensors in, torch tensors out.

Every step of the fit runs in the library's CUDA kernels; this module only
allocates outputs with PyTorch (device memory), passes pointers and the
current stream, and checks return codes.
"""

import ctypes
from dataclasses import dataclass, field

import torch

from . import _lib as L


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


class Handle:
    """A library handle bound to a CUDA device and (by default) torch's
    current stream on it."""

    def __init__(self, device=None, stream=None):
        self.lib = L.load()
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if dev.type != "cuda":
            raise ValueError("gmgm needs a CUDA device")
        self.device = dev
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        self.stream = stream
        h = ctypes.c_void_p()
        rc = self.lib.gmgm_create(ctypes.byref(h), dev.index or 0, ctypes.c_void_p(stream.cuda_stream))
        if rc != 0:
            raise L.GmgmError(rc, "gmgm_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.gmgm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def check(self, rc):
        if rc != 0:
            msg = self.lib.gmgm_last_error(self.h).decode()
            raise L.GmgmError(rc, msg)

    def device_status(self):
        """Synchronise and return (and clear) the device status bits."""
        rc = self.lib.gmgm_device_status(self.h)
        if rc < 0:
            self.check(rc)
        return rc

    def probe_wait(self, spins):
        """Enqueue the bounded-wait check (gmgm_probe_wait): a wait on a flag
        nothing sets gives up after `spins` polls and sets the TIMEOUT bit."""
        self.check(self.lib.gmgm_probe_wait(self.h, int(spins)))


_default = {}


def handle(device=None) -> Handle:
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    key = (dev.index or 0, torch.cuda.current_stream(dev).cuda_stream)
    h = _default.get(key)
    if h is None:
        h = Handle(dev)
        _default[key] = h
    return h


def _need_cuda(t, dtype, name):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}")


# ---- preprocessing ----------------------------------------------------------

def preprocess(counts: torch.Tensor, split: bool = True, inplace: bool = False, x_out: bool = True,
               h: Handle = None):
    """log1p + column centring of an n x p FP32 count matrix on the GPU.
    Returns (X, xt_hi, xt_lo, ld_t); xt_* are p x ld_t BF16 planes of X^T
    (None when split=False).  With split and x_out=False only the planes are
    written and X is None (the tensor-core Gram and lift read nothing else)."""
    h = h or handle(counts.device)
    _need_cuda(counts, torch.float32, "counts")
    if counts.dim() != 2 or counts.stride(1) != 1:
        raise ValueError("counts must be a row-major 2-D tensor")
    if not x_out and not split:
        raise ValueError("x_out=False needs split=True")
    n, p = counts.shape
    x = None if not x_out else (counts if inplace else torch.empty_like(counts))
    hi = lo = None
    ld_t = 0
    if split:
        ld_t = ((n + 63) // 64) * 64
        hi = torch.empty(p, ld_t, dtype=torch.bfloat16, device=counts.device)
        lo = torch.empty(p, ld_t, dtype=torch.bfloat16, device=counts.device)
    h.check(h.lib.gmgm_preprocess(h.h, n, p, _ptr(counts), counts.stride(0), _ptr(x),
                                  x.stride(0) if x is not None else p, _ptr(hi), _ptr(lo), ld_t, None))
    return x, hi, lo, ld_t


def preprocess_csr(indptr: torch.Tensor, indices: torch.Tensor, data: torch.Tensor, n: int, p: int,
                   h: Handle = None):
    """log1p + column centring of a CSR count matrix (n x p: int64 row
    offsets, int32 ascending column indices, FP32 counts, on the GPU) straight
    into the BF16 planes of X^T.  Returns (xt_hi, xt_lo, ld_t, column means
    FP64)."""
    h = h or handle(data.device)
    _need_cuda(indptr, torch.int64, "indptr")
    _need_cuda(indices, torch.int32, "indices")
    _need_cuda(data, torch.float32, "data")
    ld_t = ((n + 63) // 64) * 64
    hi = torch.empty(p, ld_t, dtype=torch.bfloat16, device=data.device)
    lo = torch.empty(p, ld_t, dtype=torch.bfloat16, device=data.device)
    mu = torch.empty(p, dtype=torch.float64, device=data.device)
    h.check(h.lib.gmgm_preprocess_csr(h.h, n, p, _ptr(indptr.contiguous()), _ptr(indices.contiguous()),
                                      _ptr(data.contiguous()), _ptr(hi), _ptr(lo), ld_t, _ptr(mu)))
    return hi, lo, ld_t, mu


# ---- rank-based statistics (Nonparanormal Skeptic, COCA form) ----------------

def skeptic(counts: torch.Tensor, axis: int, z: bool = True, planes: bool = True, ranks: bool = False,
            h: Handle = None):
    """Normal scores Phi^-1(rank / (N + 1)) of the ranks of a count matrix
    (n x p FP32 on the GPU) along ``axis`` (AXIS_ROWS: each row over its p
    entries; AXIS_COLS: each column over its n entries), ties at the lowest
    rank.  Returns (Z n x p FP32 or None, zt_hi, zt_lo (p x ld_t BF16 split
    of Z^T) or None, ld_t, ranks n x p int32 or None)."""
    h = h or handle(counts.device)
    _need_cuda(counts, torch.float32, "counts")
    if counts.dim() != 2 or counts.stride(1) != 1:
        raise ValueError("counts must be a row-major 2-D tensor")
    n, p = counts.shape
    dev = counts.device
    if axis == L.AXIS_ROWS and planes:
        z = True
    zt = torch.empty(n, p, dtype=torch.float32, device=dev) if z else None
    ld_t = ((n + 63) // 64) * 64 if planes else 0
    hi = torch.empty(p, ld_t, dtype=torch.bfloat16, device=dev) if planes else None
    lo = torch.empty(p, ld_t, dtype=torch.bfloat16, device=dev) if planes else None
    rk = torch.empty(n, p, dtype=torch.int32, device=dev) if ranks else None
    h.check(h.lib.gmgm_skeptic(h.h, n, p, _ptr(counts), counts.stride(0), axis, _ptr(zt), p, _ptr(hi), _ptr(lo),
                               ld_t, _ptr(rk), p))
    return zt, hi, lo, ld_t, rk


# ---- Gram ------------------------------------------------------------------

def _matrix(x=None, xt_hi=None, xt_lo=None, ld_t=0, rows=None, cols=None, batch=1, batch_stride=0):
    m = L.Matrix()
    if x is not None:
        if x.dim() == 2:
            rows, cols = x.shape
            m.ld = x.stride(0)
        elif x.dim() == 3:
            batch, rows, cols = x.shape
            m.ld = x.stride(1)
            batch_stride = x.stride(0)
        else:
            raise ValueError("x must be 2-D or 3-D")
        if x.stride(-1) != 1:
            raise ValueError("x must have unit stride in its last dimension")
        m.x = x.data_ptr()
    m.batch, m.rows, m.cols, m.batch_stride = batch, rows, cols, batch_stride
    m.xt_hi = xt_hi.data_ptr() if xt_hi is not None else None
    m.xt_lo = xt_lo.data_ptr() if xt_lo is not None else None
    m.ld_t = ld_t
    return m


def gram(x: torch.Tensor = None, side: int = L.SIDE_COLS, prec: int = L.FP32, xt_hi=None, xt_lo=None,
         ld_t: int = 0, rows: int = None, cols: int = None, out: torch.Tensor = None, accumulate=False,
         h: Handle = None):
    """S = sum_b X_b^T X_b (side COLS) or sum_b X_b X_b^T (side ROWS), FP64."""
    dev = x.device if x is not None else xt_hi.device
    h = h or handle(dev)
    if x is not None:
        _need_cuda(x, torch.float32, "x")
    m = _matrix(x, xt_hi, xt_lo, ld_t, rows, cols)
    d = m.cols if side == L.SIDE_COLS else m.rows
    if out is None:
        out = torch.empty(d, d, dtype=torch.float64, device=dev)
    h.check(h.lib.gmgm_gram(h.h, ctypes.byref(m), side, prec, _ptr(out), out.stride(0), int(accumulate)))
    return out


# ---- spectra ---------------------------------------------------------------

def spectra(S: torch.Tensor, r: int, vectors: bool = True, rv: int = None, h: Handle = None):
    """The r largest eigenvalues (descending) of a symmetric FP64 matrix on
    the GPU and the eigenvectors of the rv largest (rv = r when vectors,
    else 0)."""
    h = h or handle(S.device)
    _need_cuda(S, torch.float64, "S")
    if S.stride(1) != 1:
        S = S.contiguous()
    d = S.shape[0]
    rv = (r if vectors else 0) if rv is None else rv
    ev = torch.empty(r, dtype=torch.float64, device=S.device)
    W = torch.empty(d, rv, dtype=torch.float64, device=S.device) if rv > 0 else None
    h.check(h.lib.gmgm_spectra(h.h, d, _ptr(S), S.stride(0), r, _ptr(ev), rv, _ptr(W), max(rv, 1)))
    return ev, W


def lift(x: torch.Tensor, W: torch.Tensor, E: torch.Tensor, r: int, xt_hi=None, xt_lo=None, ld_t: int = 0,
         rows: int = None, h: Handle = None):
    """U = X W_r diag(E_r)^-1/2 (rows x r, FP32).  With the BF16 planes of
    X^T (xt_hi, xt_lo, ld_t) and r <= 64 it runs on the tensor cores from
    them (3xBF16); otherwise from X in FP32."""
    dev = x.device if x is not None else xt_hi.device
    h = h or handle(dev)
    if x is not None:
        _need_cuda(x, torch.float32, "x")
    W = W.contiguous()
    E = E.contiguous()
    if x is None and rows is None:
        raise ValueError("without x, give the number of rows")
    m = _matrix(x, xt_hi, xt_lo, ld_t, rows=rows, cols=W.shape[0])
    U = torch.empty(m.rows, r, dtype=torch.float32, device=dev)
    h.check(h.lib.gmgm_lift(h.h, ctypes.byref(m), r, _ptr(W), W.stride(0), _ptr(E), _ptr(U), r))
    return U


# ---- eigenvalue solve --------------------------------------------------------

def eigsolve(E, modalities=None, eps=None, init=None, tol=1e-9, max_newton=200, max_cg=200,
             fp32_phase=True, gauge=True, trace_rtol=0.0, h: Handle = None):
    """Eigenvalues Lam_l of the MLE.  E: list of FP64 CUDA tensors (descending
    spectra); modalities: list of tuples of axis indices (default: one
    modality over all axes).  Returns (list of FP64 tensors, stats dict)."""
    E = [e.contiguous() for e in E]
    dev = E[0].device
    h = h or handle(dev)
    for e in E:
        _need_cuda(e, torch.float64, "E")
    if modalities is None:
        modalities = [tuple(range(len(E)))]
    p = L.Problem()
    p.n_axes = len(E)
    for a, e in enumerate(E):
        p.r[a] = e.numel()
        p.E[a] = e.data_ptr()
        p.eps[a] = eps[a] if eps is not None else 0.0
    p.n_modalities = len(modalities)
    for g, m in enumerate(modalities):
        p.mod_n_axes[g] = len(m)
        for q, a in enumerate(m):
            p.mod_axes[g][q] = a
    outs = [torch.empty_like(e) for e in E]
    out_arr = (ctypes.c_void_p * len(E))(*[o.data_ptr() for o in outs])
    init_arr = None
    if init is not None:
        init = [t.contiguous() for t in init]
        init_arr = (ctypes.c_void_p * len(E))(*[t.data_ptr() for t in init])
    o = L.SolveOpts(tol, max_newton, max_cg, int(fp32_phase), int(gauge), float(trace_rtol))
    st = L.SolveStats()
    rc = h.lib.gmgm_eigsolve(h.h, ctypes.byref(p), init_arr, ctypes.byref(o), out_arr, ctypes.byref(st))
    if rc not in (0, -5):
        h.check(rc)
    return outs, st.as_dict()


# ---- top-k network -------------------------------------------------------------

def topk_network(V: torch.Tensor, psi: torch.Tensor, k: int, prec: int = L.FP32, ortho: bool = False,
                 h: Handle = None):
    """Per-row top-k of |V diag(psi) V^T| (diagonal excluded).  ortho: V is
    square with orthonormal columns (GMGM_TOPK_ORTHO).  Returns
    (idx int32 [d, k], val float32 [d, k], stats dict)."""
    h = h or handle(V.device)
    if V.dtype not in (torch.float32, torch.float64) or not V.is_cuda:
        raise ValueError("V must be a CUDA FP32/FP64 matrix")
    if V.stride(1) != 1:
        V = V.contiguous()
    _need_cuda(psi, torch.float64, "psi")
    d, r = V.shape
    idx = torch.empty(d, k, dtype=torch.int32, device=V.device)
    val = torch.empty(d, k, dtype=torch.float32, device=V.device)
    st = L.TopkStats()
    h.check(h.lib.gmgm_topk_network(h.h, d, r, _ptr(V), int(V.dtype == torch.float64), V.stride(0),
                                    _ptr(psi.contiguous()), k, prec, L.TOPK_ORTHO if ortho else 0, _ptr(idx),
                                    _ptr(val), ctypes.byref(st)))
    return idx, val, st.as_dict()


def topk_network_rows(V: torch.Tensor, psi: torch.Tensor, k: int, row0: int, m: int, prec: int = L.FP32,
                      h: Handle = None):
    """Rows [row0, row0 + m) of the network of topk_network (every column
    screened): idx int32 [m, k], val float32 [m, k], stats dict."""
    h = h or handle(V.device)
    if V.dtype not in (torch.float32, torch.float64) or not V.is_cuda:
        raise ValueError("V must be a CUDA FP32/FP64 matrix")
    if V.stride(1) != 1:
        V = V.contiguous()
    _need_cuda(psi, torch.float64, "psi")
    d, r = V.shape
    idx = torch.empty(m, k, dtype=torch.int32, device=V.device)
    val = torch.empty(m, k, dtype=torch.float32, device=V.device)
    st = L.TopkStats()
    h.check(h.lib.gmgm_topk_network_rows(h.h, d, r, _ptr(V), int(V.dtype == torch.float64), V.stride(0),
                                         _ptr(psi.contiguous()), k, prec, row0, m, _ptr(idx), _ptr(val),
                                         ctypes.byref(st)))
    return idx, val, st.as_dict()


def topk_network_gram(S: torch.Tensor, psi: torch.Tensor, k: int, prec: int = L.FP32, h: Handle = None):
    """Network of a full-rank axis from its Gram S: top-k of |W diag(psi) W^T|
    with W the eigenvectors of S (psi in descending eigenvalue order); only
    the eigenvectors whose psi exceeds min psi are formed."""
    h = h or handle(S.device)
    _need_cuda(S, torch.float64, "S")
    if S.stride(1) != 1:
        S = S.contiguous()
    _need_cuda(psi, torch.float64, "psi")
    d = S.shape[0]
    idx = torch.empty(d, k, dtype=torch.int32, device=S.device)
    val = torch.empty(d, k, dtype=torch.float32, device=S.device)
    st = L.TopkStats()
    h.check(h.lib.gmgm_topk_network_gram(h.h, d, _ptr(S), S.stride(0), _ptr(psi.contiguous()), k, prec, _ptr(idx),
                                         _ptr(val), ctypes.byref(st)))
    return idx, val, st.as_dict()


def topn_edges(idx: torch.Tensor, val: torch.Tensor, n: int, h: Handle = None):
    """Global top-n edges (i < j) from per-row top-k lists (d x k int32 /
    FP32 on the GPU).  Returns (i, j, value, certified): the union's n
    strongest pairs by |value| descending then (i, j), and whether they are
    certified to be the network's global top-n."""
    h = h or handle(idx.device)
    _need_cuda(idx, torch.int32, "idx")
    _need_cuda(val, torch.float32, "val")
    idx, val = idx.contiguous(), val.contiguous()
    d, k = idx.shape
    io = torch.empty(n, dtype=torch.int32, device=idx.device)
    jo = torch.empty(n, dtype=torch.int32, device=idx.device)
    vo = torch.empty(n, dtype=torch.float32, device=idx.device)
    cnt = ctypes.c_int64(0)
    cert = ctypes.c_int(0)
    h.check(h.lib.gmgm_topn_edges(h.h, d, k, _ptr(idx), _ptr(val), n, _ptr(io), _ptr(jo), _ptr(vo),
                                  ctypes.byref(cnt), ctypes.byref(cert)))
    c = cnt.value
    return io[:c], jo[:c], vo[:c], bool(cert.value)


# ---- the whole two-axis fit -----------------------------------------------------

@dataclass
class TwoAxisResult:
    e_rows: torch.Tensor
    v_rows: torch.Tensor
    e_cols: torch.Tensor
    v_cols: torch.Tensor      # None when the gene axis is at full rank (not formed)
    lam_rows: torch.Tensor
    lam_cols: torch.Tensor
    idx_rows: torch.Tensor
    val_rows: torch.Tensor
    idx_cols: torch.Tensor
    val_cols: torch.Tensor
    solve: dict = field(default_factory=dict)
    topk_rows_stats: dict = field(default_factory=dict)
    topk_cols_stats: dict = field(default_factory=dict)
    s_cols: torch.Tensor = None  # the gene Gram X^T X (FP64)


def fit_two_axis(x: torch.Tensor, r_rows: int, r_cols: int, k_rows: int, k_cols: int,
                 gram_prec: int = L.FP32, topk_prec: int = L.FP32, xt_hi=None, xt_lo=None, ld_t=0,
                 tol: float = 1e-9, fp32_phase=True, init=None, warm_params=None, rows: int = None,
                 h: Handle = None) -> TwoAxisResult:
    """Algorithm 1 on a centred matrix X (rows x cols, FP32, on the GPU):
    S_cols = X^T X, its eigenpairs (FP64), the row-axis vectors by the dual
    lift, the eigenvalue solve (from `init`, or from the learned start when
    `warm_params` is given, else from 1/E), and both per-row top-k networks.
    x may be None when the BF16 planes of X^T are given (with `rows`), e.g.
    from preprocess_csr."""
    dev = x.device if x is not None else xt_hi.device
    h = h or handle(dev)
    n = x.shape[0] if x is not None else rows
    p = x.shape[1] if x is not None else xt_hi.shape[0]
    S = gram(x, L.SIDE_COLS, gram_prec, xt_hi=xt_hi, xt_lo=xt_lo, ld_t=ld_t, rows=n, cols=p, h=h)
    rmax = max(r_rows, r_cols)
    full = r_cols == S.shape[0]
    # eigenvectors: the cell axis' r_rows for the lift; the gene axis' only
    # when it is truncated (at full rank its network comes from S directly)
    ev, W = spectra(S, rmax, rv=r_rows if full else rmax, h=h)
    e_cols = ev[:r_cols].contiguous()
    v_cols = None if full else W[:, :r_cols].contiguous()
    e_rows = ev[:r_rows].contiguous()
    if init is None and warm_params is not None:
        i0, i1 = torch.empty_like(e_rows), torch.empty_like(e_cols)
        h.check(h.lib.gmgm_warmstart_infer(h.h, _ptr(warm_params), _ptr(e_rows), r_rows, _ptr(e_cols), r_cols,
                                           0.0, _ptr(i0), _ptr(i1)))
        init = [i0, i1]
    v_rows = lift(x, W[:, :r_rows].contiguous(), e_rows, r_rows, xt_hi=xt_hi, xt_lo=xt_lo, ld_t=ld_t, rows=n, h=h)
    (lam_rows, lam_cols), st = eigsolve([e_rows, e_cols], [(0, 1)], tol=tol, fp32_phase=fp32_phase,
                                        init=init, h=h)
    ir, vr, sr = topk_network(v_rows, lam_rows, k_rows, topk_prec, h=h)
    if full:
        ic, vc, sc = topk_network_gram(S, lam_cols, k_cols, L.FP32, h=h)
    else:
        ic, vc, sc = topk_network(v_cols, lam_cols, k_cols, L.FP32, h=h)
    return TwoAxisResult(e_rows, v_rows, e_cols, v_cols, lam_rows, lam_cols, ir, vr, ic, vc, st, sr, sc, S)


def fit_two_axis_skeptic(counts: torch.Tensor, r_rows: int, k_rows: int, k_cols: int, tol: float = 1e-9,
                         h: Handle = None) -> TwoAxisResult:
    """Algorithm 1 on rank-based statistics (Section "The model": the
    Nonparanormal Skeptic; Section "Algorithm": its COCA form) of a count
    matrix (cells x genes, FP32, on the GPU).  Each axis' Gram is the Gram of
    its own normal scores: S_genes = Z_g^T Z_g with Z_g the scores of every
    gene ranked over the cells; the cell axis from Z_c, every cell ranked over
    its genes, through the dual Gram Z_c^T Z_c (its top r_rows eigenpairs)
    and the lift U = Z_c W diag(E)^-1/2.  Then the solve (E_cells the top
    eigenvalues, E_genes the full gene spectrum) and both networks.  Grams
    in 3xBF16, the cell screen in BF16 (as the log1p fit)."""
    h = h or handle(counts.device)
    n, p = counts.shape
    _, ghi, glo, ld_t, _ = skeptic(counts, L.AXIS_COLS, z=False, planes=True, h=h)
    Sg = gram(None, L.SIDE_COLS, L.BF16X3, xt_hi=ghi, xt_lo=glo, ld_t=ld_t, rows=n, cols=p, h=h)
    del ghi, glo
    zc, chi, clo, ld_t, _ = skeptic(counts, L.AXIS_ROWS, planes=True, h=h)
    del zc
    Sc = gram(None, L.SIDE_COLS, L.BF16X3, xt_hi=chi, xt_lo=clo, ld_t=ld_t, rows=n, cols=p, h=h)
    e_rows, Wc = spectra(Sc, r_rows, rv=r_rows, h=h)
    U = lift(None, Wc, e_rows, r_rows, xt_hi=chi, xt_lo=clo, ld_t=ld_t, rows=n, h=h)
    del chi, clo
    e_cols, _ = spectra(Sg, p, vectors=False, h=h)
    (lam_rows, lam_cols), st = eigsolve([e_rows, e_cols], [(0, 1)], tol=tol, h=h)
    ir, vr, sr = topk_network(U, lam_rows, k_rows, L.BF16, h=h)
    ic, vc, sc = topk_network_gram(Sg, lam_cols, k_cols, L.FP32, h=h)
    return TwoAxisResult(e_rows, U, e_cols, None, lam_rows, lam_cols, ir, vr, ic, vc, st, sr, sc, Sg)


# ---- several modalities sharing the cell axis; one K-axis tensor ---------------

@dataclass
class MultiAxisResult:
    E: list        # per axis, FP64 descending
    V: list        # per axis, eigenvectors as columns (cells: FP32 lift); None for a full-rank
                   # axis, whose network comes from its Gram
    S: list        # per axis, the Gram its spectrum and network come from (cells: the Gram of the
                   # concatenation; a feature axis: its diagonal block)
    lam: list      # per axis, FP64
    idx: list      # per axis, int32 [d_l, k_l] (None where no network was asked)
    val: list      # per axis, FP32 [d_l, k_l]
    solve: dict = field(default_factory=dict)
    topk_stats: list = field(default_factory=list)


def fit_multimodal(counts, r_cells: int, ks, gram_prec: int = L.BF16X3, topk_prec: int = L.BF16,
                   tol: float = 1e-9, h: Handle = None) -> MultiAxisResult:
    """Count matrices (cells x p_m, FP32, on the GPU) sharing the cell axis.

    Section "Algorithm": the Gram of an axis shared by several modalities is
    the Gram of their concatenation.  Each modality is preprocessed into its
    column slice of one X = [X_1 X_2 ...] (and its rows of the BF16 planes of
    X^T); one column Gram of X holds every block.  The cell axis takes the top
    r_cells eigenpairs of that Gram lifted through X; modality m's own axis
    takes the full spectrum of its diagonal block.  The solve couples
    (cells, m) for every modality; one network per axis (ks: k per axis,
    cells first)."""
    dev = counts[0].device
    h = h or handle(dev)
    n = counts[0].shape[0]
    ps = [c.shape[1] for c in counts]
    P = sum(ps)
    for c in counts:
        _need_cuda(c, torch.float32, "counts")
        if c.dim() != 2 or c.shape[0] != n or c.stride(1) != 1:
            raise ValueError("every count matrix must be row-major cells x features with the same cells")
    split = gram_prec != L.FP32
    # with the BF16 planes (and r_cells <= 64, the tensor-core lift) the FP32 X is never read: not written
    x = None if split and r_cells <= 64 else torch.empty(n, P, dtype=torch.float32, device=dev)
    ld_t = ((n + 63) // 64) * 64 if split else 0
    hi = torch.empty(P, ld_t, dtype=torch.bfloat16, device=dev) if split else None
    lo = torch.empty(P, ld_t, dtype=torch.bfloat16, device=dev) if split else None
    off = 0
    for c, p in zip(counts, ps):
        h.check(h.lib.gmgm_preprocess(h.h, n, p, _ptr(c), c.stride(0), _ptr(x[:, off:]) if x is not None else None,
                                      x.stride(0) if x is not None else p,
                                      _ptr(hi[off:]) if split else None, _ptr(lo[off:]) if split else None,
                                      ld_t, None))
        off += p
    S = gram(x, L.SIDE_COLS, gram_prec, xt_hi=hi, xt_lo=lo, ld_t=ld_t, rows=n, cols=P, h=h)
    e_c, W_c = spectra(S, r_cells, True, h=h)
    E, V, Ss = [e_c], [lift(x, W_c, e_c, r_cells, xt_hi=hi, xt_lo=lo, ld_t=ld_t, rows=n, h=h)], [S]
    off = 0
    for p in ps:
        Sb = S[off:off + p, off:off + p]
        e, _ = spectra(Sb, p, vectors=False, h=h)
        E.append(e)
        V.append(None)
        Ss.append(Sb)
        off += p
    lams, st = eigsolve(E, [(0, m + 1) for m in range(len(ps))], tol=tol, h=h)
    idx, val, sts = [], [], []
    for a in range(len(E)):
        if ks[a]:
            if a == 0:
                i, v, t = topk_network(V[0], lams[0], ks[0], topk_prec, h=h)
            else:  # a feature axis at full rank
                i, v, t = topk_network_gram(Ss[a], lams[a], ks[a], L.FP32, h=h)
        else:
            i = v = t = None
        idx.append(i)
        val.append(v)
        sts.append(t)
    return MultiAxisResult(E, V, Ss, lams, idx, val, st, sts)


def fit_tensor(t: torch.Tensor, ks, tol: float = 1e-9, h: Handle = None) -> MultiAxisResult:
    """One 3-axis tensor T (d0 x d1 x d2, FP32, row-major, on the GPU): the
    Gram of every axis (Notation: S_l = mat_l[T] mat_l[T]^T), its full FP64
    spectrum, the solve over one modality of all three axes, and one network
    per axis (ks: k per axis, None for none)."""
    h = h or handle(t.device)
    _need_cuda(t, torch.float32, "t")
    if t.dim() != 3:
        raise ValueError("t must be a 3-axis tensor")
    t = t.contiguous()
    d0, d1, d2 = t.shape
    Ss = [gram(t.reshape(d0, d1 * d2), L.SIDE_ROWS, L.FP32, h=h),
          gram(t, L.SIDE_ROWS, L.FP32, h=h),
          gram(t.reshape(d0 * d1, d2), L.SIDE_COLS, L.FP32, h=h)]
    E = [spectra(S, S.shape[0], vectors=False, h=h)[0] for S in Ss]
    lams, st = eigsolve(E, [(0, 1, 2)], tol=tol, h=h)
    idx, val, sts = [], [], []
    for a in range(3):
        if ks[a]:
            i, v, s_ = topk_network_gram(Ss[a], lams[a], ks[a], L.FP32, h=h)
        else:
            i = v = s_ = None
        idx.append(i)
        val.append(v)
        sts.append(s_)
    return MultiAxisResult(E, [None] * 3, Ss, lams, idx, val, st, sts)
