"""B300-native (sm_103a) DINR training step and query server.

The compute path is libdinr.so (hand-written CUDA behind a C ABI,
include/dinr.h); this package is its Python binding.
"""
from .dinr import (Dinr, DinrError, DinrStep, param_count, param_count_net,  # noqa: F401
                   phantom_project)
