"""Upscaled-field error of every benchmark workload against the FP64 oracle.

Each case runs the GPU on a whole batch of the workload's boxes (in the launch
configuration the benchmark times) and the oracle on sampled boxes: the first,
the last, the largest and smallest of uneven batches and a seeded random pick.
The error measure and bounds are those of test_gpu_parity.py (1e-6 relative
for the batched FP32 form, 1e-12 for the FP64 method against the oracle in long
double). The 3D workload runs at its full 64^3 macro grid (262,144 boxes of
32^3, 300 steps; the FP32 form on the whole batch, the FP64 method through
hmm_micro_batch_points on its sampled box) and on a 16^3 macro grid; the
micro-solver sweep runs 1k-box batches at each box size and micro damping of
the sweep, the FP64 method at all twelve points. Where the long-double oracle
would take minutes on the test machine (one 128^2 or 32^3 box), its values are
read from tests/golden/longdouble_refs.json, written once by
tests/golden/make_longdouble_refs.py from the oracle.

With HMM_PARITY_REPORT=<file> set, each case appends one JSON line (workload,
precision, kernel, sampled boxes, error) to that file.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import hmm_oracle as O

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-6}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_09463_gb300 import build
    build()
    return torch


def rel_err(Hg, Hr):
    d = (np.asarray(Hg, dtype=Hr.dtype) - Hr).astype(np.float64)
    return np.linalg.norm(d, axis=0).max() / np.linalg.norm(Hr.astype(np.float64), axis=0).max()


def _report(rec):
    path = os.environ.get("HMM_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(rec) + "\n")


# name -> (workload, overrides, FP32 sample size, FP64 sample size)
CASES = {
    "c1_1d": ("c1_1d", {}, 64, 4),
    "c2_2d": ("c2_2d", {}, 6, 2),
    "c3_2d_uneven": ("c3_2d_uneven", {}, 6, 2),
    "c4_3d_sub16": ("c4_3d", dict(n_macro=(16, 16, 16)), 4, 1),
    "c4_3d_full": ("c4_3d", {}, 4, 1),
}
for _n in (48, 64, 96, 128):
    for _a in (0.01, 0.1, 1.0):
        CASES[f"c5_N{_n}_a{_a:g}"] = ("c5_sweep", dict(box_n=_n, alpha_micro=_a), 3, 1)

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "longdouble_refs.json")


def _golden(case):
    with open(GOLDEN) as f:
        return json.load(f)["cases"].get(case)


def _points(cfg, N, k, seed, small_first):
    """k boxes: the largest and smallest boxes, the first and last, then random ones.
    small_first puts the smallest box first (the long-double oracle is slow)."""
    P = cfg.n_points
    if k >= P:
        return list(range(P))
    order = [int(np.argmin(N)), int(np.argmax(N))] if small_first else [int(np.argmax(N)), int(np.argmin(N))]
    pts = []
    for p in order + [0, P - 1]:
        if p not in pts and len(pts) < k:
            pts.append(p)
    rng = np.random.default_rng(seed)
    while len(pts) < k:
        p = int(rng.integers(P))
        if p not in pts:
            pts.append(p)
    return sorted(pts)


@pytest.mark.parametrize("precision", [1, 0], ids=["fp32", "fp64"])
@pytest.mark.parametrize("case", list(CASES))
def test_workload_error(torch_cuda, case, precision):
    from paper_2108_09463_gb300 import HMM
    name, over, k32, k64 = CASES[case]
    k = k32 if precision == 1 else k64
    cfg = W.config(name, **over)
    M0 = W.initial_field(cfg)
    h = HMM(cfg, precision=precision)
    M = torch_cuda.from_numpy(M0).cuda()
    gold = _golden(case) if precision == 0 else None
    if gold is not None:
        assert gold["workload"] == name and gold["overrides"] == {kk: v for kk, v in over.items()}
        pts = list(gold["points"])
        # the sampled boxes only (the whole FP64 batch of the 3D workload would take minutes)
        Hg = h.micro_batch_points(M, pts).cpu().numpy()
        Hr = np.array(gold["H"], dtype=np.float64)
    else:
        Hg = h.micro_batch(M).cpu().numpy()
    info = h.box_info()
    lu, ms = h.stats()
    h.close()
    if gold is None:
        assert np.all(np.isfinite(Hg))
        pts = _points(cfg, info["N"], k, seed=7, small_first=precision == 0)
        dtype = np.longdouble if precision == 0 else np.float64
        Hr = O.micro_batch(cfg, M0, points=pts, dtype=dtype)
    e = float(rel_err(Hg[:, pts], Hr))
    _report(dict(case=case, workload=name, precision="fp64" if precision == 0 else "fp32",
                 boxes=cfg.n_points, sampled=len(pts), N_min=int(info["N"].min()), N_max=int(info["N"].max()),
                 rel_err=e, lattice_updates=lu, batch_ms=ms, reference="golden long double" if gold else "oracle"))
    assert e < TOL[precision], (case, precision, e)
