"""GB300-native direct N-body Hermite block-step library (sm_103a CUDA).

The compute path lives in ``libnb_gb300.so`` (sources in ``csrc/``, ABI in
``include/nb.h``); ``nb`` is its Python binding.
"""
from .nb import *  # noqa: F401,F403
from .nb import Context, Ensemble, NbError, lib  # noqa: F401
