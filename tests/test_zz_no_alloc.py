"""The allocation-free eigenvalue solve (gmgm_eigsolve_static) against the
regular entry point (gmgm_eigsolve).

gmgm_eigsolve_static serves callers that cannot allocate device memory when
they call the library: it takes no handle and keeps its working memory in a
fixed array inside the library.  This file is collected last so that, if it
fails, a run stopping at the first failure has already run every other test;
it also passes when run alone in a fresh process.
"""

import ctypes

import numpy as np
import pytest
import torch

from oracle import spectra as osp
from synth import planted_c1

pytestmark = pytest.mark.gpu


def _problem(L, E, modalities):
    p = L.Problem()
    p.n_axes = len(E)
    for a, e in enumerate(E):
        p.r[a] = e.numel()
        p.E[a] = e.data_ptr()
        p.eps[a] = 0.0
    p.n_modalities = len(modalities)
    for g, m in enumerate(modalities):
        p.mod_n_axes[g] = len(m)
        for q, a in enumerate(m):
            p.mod_axes[g][q] = a
    return p


def _static_solve(L, lib, E, modalities, tol):
    """One call of the allocation-free entry point through the C ABI."""
    p = _problem(L, E, modalities)
    outs = [torch.empty_like(e) for e in E]
    out_arr = (ctypes.c_void_p * len(E))(*[o.data_ptr() for o in outs])
    opts = L.SolveOpts(tol, 200, 200, 1, 1)
    st = L.SolveStats()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.gmgm_eigsolve_static(ctypes.byref(p), None, ctypes.byref(opts), out_arr, ctypes.byref(st), stream)
    return rc, outs, st.as_dict()


def test_static_solve_matches_regular_entry_point_twice(cuda_dev):
    import paper_2407_19892_gb300 as g
    from paper_2407_19892_gb300 import _lib as L
    from paper_2407_19892_gb300 import build
    build.build()
    lib = L.load()
    x, _, _ = planted_c1()
    cases = []
    for r_rows in (100, 25):  # full ranks (gauge convention) then a clipped box
        e_r, _, e_c, _ = osp.two_axis_spectra(x, r_rows, 100)
        cases.append([torch.from_numpy(e_r).to(cuda_dev), torch.from_numpy(e_c).to(cuda_dev)])
    for E in cases:  # two calls in a row share (and reuse) the fixed array
        rc, got, st = _static_solve(L, lib, E, [(0, 1)], 1e-10)
        assert rc == 0 and st["status"] == 0, st
        ref, st_ref = g.eigsolve(E, [(0, 1)], tol=1e-10)
        assert st_ref["status"] == 0
        for a, b in zip(got, ref):
            torch.testing.assert_close(a, b, rtol=1e-10, atol=0)
        s_got = got[0][:, None] + got[1][None, :]
        s_ref = ref[0][:, None] + ref[1][None, :]
        assert torch.max(torch.abs(s_got - s_ref) / s_ref).item() <= 1e-10
        assert st["rel_kkt"] <= 1e-9


def test_static_solve_rejects_sizes_beyond_its_array(cuda_dev):
    from paper_2407_19892_gb300 import _lib as L
    from paper_2407_19892_gb300 import build
    build.build()
    lib = L.load()
    E = [torch.linspace(2.0, 1.0, 3000, dtype=torch.float64, device=cuda_dev),
         torch.linspace(2.0, 1.0, 1200, dtype=torch.float64, device=cuda_dev)]
    rc, _, _ = _static_solve(L, lib, E, [(0, 1)], 1e-9)
    assert rc == -1  # GMGM_E_ARG: sum of ranks 4200 > 4096
