"""ctypes binding of libgmgm (include/gmgm.h): argument marshalling only.

The library must have been built (``paper_2407_19892_gb300.build.build()``);
loading fails loudly otherwise.  There is no fallback implementation.
"""

import ctypes
import os

from .build import LIB

c_int = ctypes.c_int
c_i32 = ctypes.c_int32
c_i64 = ctypes.c_int64
c_dbl = ctypes.c_double
c_vp = ctypes.c_void_p

GMGM_OK = 0
STATUS = {0: "GMGM_OK", -1: "GMGM_E_ARG", -2: "GMGM_E_CUDA", -3: "GMGM_E_NOMEM",
          -4: "GMGM_E_NONFINITE", -5: "GMGM_E_NOT_CONVERGED", -6: "GMGM_E_INFEASIBLE",
          -7: "GMGM_E_CAND_OVERFLOW", -8: "GMGM_E_TIMEOUT"}
FP32, BF16, BF16X3, FP64 = 0, 1, 2, 3
SIDE_COLS, SIDE_ROWS = 0, 1
AXIS_ROWS, AXIS_COLS = 0, 1
DEV_NOT_COUNTS = 0x20
MAX_AXES, MAX_MODALITIES = 4, 4


class Matrix(ctypes.Structure):
    _fields_ = [("batch", c_i64), ("rows", c_i64), ("cols", c_i64), ("ld", c_i64),
                ("batch_stride", c_i64), ("x", c_vp), ("xt_hi", c_vp), ("xt_lo", c_vp),
                ("ld_t", c_i64)]


class Problem(ctypes.Structure):
    _fields_ = [("n_axes", c_i32), ("r", c_i32 * MAX_AXES), ("E", c_vp * MAX_AXES),
                ("eps", c_dbl * MAX_AXES), ("n_modalities", c_i32),
                ("mod_n_axes", c_i32 * MAX_MODALITIES),
                ("mod_axes", (c_i32 * MAX_AXES) * MAX_MODALITIES)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", c_dbl), ("max_newton", c_i32), ("max_cg", c_i32),
                ("fp32_phase", c_i32), ("gauge", c_i32), ("trace_rtol", c_dbl)]


class SolveStats(ctypes.Structure):
    _fields_ = [("status", c_i32), ("newton_iters", c_i32), ("cg_iters", c_i32),
                ("grid_passes", c_i32), ("n_active", c_i32), ("fp64_iters", c_i32),
                ("rel_kkt", c_dbl), ("objective", c_dbl)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class TrainOpts(ctypes.Structure):
    _fields_ = [("steps", c_i32), ("batch", c_i32), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("seed", ctypes.c_uint64)]


TOPK_ORTHO = 1
MLP_IN, MLP_HIDDEN, MLP_OUT = 132, 256, 128
MLP_PARAMS = 256 * 132 + 256 + 256 * 256 + 256 + 128 * 256 + 128


class TopkStats(ctypes.Structure):
    _fields_ = [("rows_uncertified", c_i64), ("rows_exact", c_i64), ("candidates", c_i64),
                ("screen_ms", c_dbl), ("rescore_ms", c_dbl), ("screen_err_ratio", c_dbl),
                ("screen_tiles", c_i64), ("screen_tiles_dense", c_i64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# name -> (restype, argtypes); mirrors include/gmgm.h
SIGNATURES = {
    "gmgm_create": (c_int, [ctypes.POINTER(c_vp), c_int, c_vp]),
    "gmgm_destroy": (c_int, [c_vp]),
    "gmgm_set_stream": (c_int, [c_vp, c_vp]),
    "gmgm_last_error": (ctypes.c_char_p, [c_vp]),
    "gmgm_device_status": (c_int, [c_vp]),
    "gmgm_probe_wait": (c_int, [c_vp, c_i64]),
    "gmgm_version": (ctypes.c_char_p, []),
    "gmgm_kernel_launches": (ctypes.c_uint64, []),
    "gmgm_preprocess": (c_int, [c_vp, c_i64, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_vp,
                                c_i64, c_vp]),
    "gmgm_skeptic": (c_int, [c_vp, c_i64, c_i64, c_vp, c_i64, c_int, c_vp, c_i64, c_vp, c_vp, c_i64,
                             c_vp, c_i64]),
    "gmgm_gram": (c_int, [c_vp, ctypes.POINTER(Matrix), c_int, c_int, c_vp, c_i64, c_int]),
    "gmgm_spectra": (c_int, [c_vp, c_i64, c_vp, c_i64, c_i32, c_vp, c_i32, c_vp, c_i64]),
    "gmgm_lift": (c_int, [c_vp, ctypes.POINTER(Matrix), c_i32, c_vp, c_i64, c_vp, c_vp, c_i64]),
    "gmgm_eigsolve": (c_int, [c_vp, ctypes.POINTER(Problem), ctypes.POINTER(c_vp),
                              ctypes.POINTER(SolveOpts), ctypes.POINTER(c_vp),
                              ctypes.POINTER(SolveStats)]),
    "gmgm_eigsolve_static": (c_int, [ctypes.POINTER(Problem), ctypes.POINTER(c_vp),
                                     ctypes.POINTER(SolveOpts), ctypes.POINTER(c_vp),
                                     ctypes.POINTER(SolveStats), c_vp]),
    "gmgm_warmstart_features": (c_int, [c_vp, c_vp, c_i32, c_vp, c_i32, c_vp]),
    "gmgm_warmstart_targets": (c_int, [c_vp, c_vp, c_i32, c_vp, c_i32, c_vp, c_vp, c_vp]),
    "gmgm_mlp_forward": (c_int, [c_vp, c_vp, c_vp, c_i32, c_vp]),
    "gmgm_mlp_loss_grad": (c_int, [c_vp, c_vp, c_vp, c_vp, c_i32, c_vp, ctypes.POINTER(ctypes.c_float)]),
    "gmgm_warmstart_train": (c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, c_i32, ctypes.POINTER(TrainOpts),
                                     ctypes.POINTER(ctypes.c_float)]),
    "gmgm_warmstart_infer": (c_int, [c_vp, c_vp, c_vp, c_i32, c_vp, c_i32, c_dbl, c_vp, c_vp]),
    "gmgm_topk_network": (c_int, [c_vp, c_i64, c_i32, c_vp, c_int, c_i64, c_vp, c_i32, c_int,
                                  ctypes.c_uint32, c_vp, c_vp, ctypes.POINTER(TopkStats)]),
    "gmgm_topk_network_rows": (c_int, [c_vp, c_i64, c_i32, c_vp, c_int, c_i64, c_vp, c_i32, c_int, c_i64, c_i64,
                                       c_vp, c_vp, ctypes.POINTER(TopkStats)]),
    "gmgm_peak_probe": (c_int, [c_vp, c_int, c_i64, ctypes.POINTER(c_dbl)]),
    "gmgm_preprocess_csr": (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_i64, c_vp]),
    "gmgm_colsum_log1p": (c_int, [c_vp, c_i64, c_i64, c_vp, c_i64, c_vp, c_int]),
    "gmgm_centre": (c_int, [c_vp, c_i64, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_vp, c_i64]),
    "gmgm_topn_edges": (c_int, [c_vp, c_i64, c_i32, c_vp, c_vp, c_i64, c_vp, c_vp, c_vp, ctypes.POINTER(c_i64),
                                ctypes.POINTER(c_int)]),
    "gmgm_topk_network_gram": (c_int, [c_vp, c_i64, c_vp, c_i64, c_vp, c_i32, c_int, c_vp, c_vp,
                                       ctypes.POINTER(TopkStats)]),
}

_lib = None


def load(path: str = LIB):
    """Load libgmgm.so (once) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libgmgm not built ({path}); run paper_2407_19892_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class GmgmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
