"""GB300 (sm_103a) library for the HMM micro-problem path of the Landau-Lifshitz
equation (Leitenmaier & Runborg, "Heterogeneous multiscale methods for the
Landau-Lifshitz equation").

The compute lives in libhmm_gb300.so (C ABI, include/hmm.h); ``HMM`` is a thin
ctypes binding. ``build()`` compiles the library in-tree with nvcc.
"""
from ._lib import (EXPORTED, HMM, HMM_FP32_BATCHED, HMM_FP64_PLAIN, HmmError,  # noqa: F401
                   load_library, make_params, micro_batch_noalloc)
from .build import build  # noqa: F401
