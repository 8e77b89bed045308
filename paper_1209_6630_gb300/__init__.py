"""GB300-native batched all-electron QMC walker evaluation (arXiv:1209.6630).

The compute lives in libqmcgb (CUDA, sm_103a; C ABI in include/qmcgb.h);
this package is its thin PyTorch binding.
"""
from .api import (QmcSystem, QmcBatch, det_inverse, LogPsi, QmcError, dmc_move, dmc_weight,  # noqa: F401
                  srmc_reconfigure, multidet_eval)
from ._lib import lib, PREC, STATUS_SINGULAR_UP, STATUS_SINGULAR_DN, STATUS_NONFINITE  # noqa: F401
