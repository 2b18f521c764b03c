"""GB300 (sm_103a) implementation of the data-parallel core of the improved
multi-axis Gaussian graphical model fit (GmGM, arXiv 2407.19892).

The compute path is the CUDA library ``libgmgm`` (C ABI in include/gmgm.h);
this package holds its build script and a thin ctypes binding.
"""

from ._lib import (AXIS_COLS, AXIS_ROWS, BF16, BF16X3, FP32, FP64, SIDE_COLS, SIDE_ROWS,  # noqa: F401
                   GmgmError, load)
from .api import (Handle, MultiAxisResult, TwoAxisResult, eigsolve, fit_multimodal,  # noqa: F401
                  fit_tensor, fit_two_axis, fit_two_axis_skeptic, gram, handle, lift, preprocess, preprocess_csr, skeptic, spectra, topk_network,
                  topk_network_gram, topk_network_rows, topn_edges)

__version__ = "0.1.0"
