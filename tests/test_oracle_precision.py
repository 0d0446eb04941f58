"""The FP64 oracle's own rounding floor for H_avg.

H_avg is an O(1..100) average of a field that is O(1e3..1e4) pointwise and
oscillates on the eps scale, and the micro dynamics carry rounding errors of
the state forward, so the plain FP64 evaluation of the scheme (the m-form of
Section 3.1's HeunP) differs from an evaluation in long double by ~1e-12
relative. This bounds what an FP64-vs-FP64 comparison can resolve; the GPU
FP64 method is therefore compared with the long-double evaluation.
"""
import numpy as np
import pytest

import workloads as W
from oracle import hmm_oracle as O


@pytest.mark.skipif(np.finfo(np.longdouble).eps >= 1e-18, reason="needs an extended long double")
@pytest.mark.parametrize("name,over", [
    ("c2_2d", dict(n_macro=(8, 8, 1), box_n=24, micro_steps=60)),
    ("c1_1d", dict(n_macro=(16, 1, 1), box_n=81, micro_steps=120)),
])
def test_fp64_oracle_floor(name, over):
    cfg = W.config(name, **over)
    M0 = W.initial_field(cfg)
    pts = [0, 5, cfg.n_points - 1]
    H64 = O.micro_batch(cfg, M0, points=pts)
    HL = O.micro_batch(cfg, M0, points=pts, dtype=np.longdouble)
    d = (H64 - HL).astype(np.float64)
    rel = np.linalg.norm(d, axis=0).max() / np.linalg.norm(HL.astype(np.float64), axis=0).max()
    assert 1e-16 < rel < 3e-12, rel


def test_longdouble_oracle_agrees_with_fp64_oracle_to_roundoff():
    """The precision switch changes rounding only (no arithmetic difference)."""
    cfg = W.config("c2_2d", n_macro=(8, 8, 1), box_n=24, micro_steps=10)
    M0 = W.initial_field(cfg)
    H64 = O.micro_batch(cfg, M0, points=[3])
    HL = O.micro_batch(cfg, M0, points=[3], dtype=np.longdouble)
    assert np.abs((H64 - HL).astype(np.float64)).max() < 1e-9 * np.abs(H64).max()
