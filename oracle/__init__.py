"""FP64 CPU oracle of the HMM micro-problem path (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline/reference leg
may import this package. The CUDA path never does.
"""
from . import hmm_oracle  # noqa: F401
