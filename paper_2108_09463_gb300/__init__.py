"""GB300 (sm_103a) library for the HMM micro-problem path of the Landau-Lifshitz
equation (Leitenmaier & Runborg, "Heterogeneous multiscale methods for the
Landau-Lifshitz equation").

The compute lives in libhmm_gb300.so (C ABI, include/hmm.h and
include/hmm_dns.h); ``HMM`` and ``DNS`` are thin ctypes bindings. ``build()`` compiles the library in-tree with nvcc.
"""
from ._lib import (DNS, EXPORTED, EXPORTED_DNS, HMM, HMM_FP32_BATCHED, HMM_FP64_PLAIN,  # noqa: F401
                   HmmError, fp32_fma_rate, load_library, make_dns_params, make_params, micro_batch_noalloc)
from .build import build  # noqa: F401
