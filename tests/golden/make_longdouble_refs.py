"""Write tests/golden/longdouble_refs.json: the oracle's H_avg in long double.

The FP64 GPU method is held to 1e-12 relative against the oracle evaluated in
long double (two FP64 evaluations of this average already differ by about
2e-12). On the GPU machine numpy's long double is IEEE quad, evaluated in software
and too slow for one 128^2 or 32^3 box per test; this script evaluates the same
oracle once (x86 80-bit extended here) and stores the values. It calls only
oracle/ and the seeded input generators of workloads/.

    python tests/golden/make_longdouble_refs.py
"""
import json
import multiprocessing as mp
import os
import platform
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "longdouble_refs.json")

# name -> (workload, overrides, macro points)
CASES = {}
for _n in (48, 64, 96, 128):
    for _a in (0.01, 0.1, 1.0):
        CASES[f"c5_N{_n}_a{_a:g}"] = ("c5_sweep", dict(box_n=_n, alpha_micro=_a), [0])
# the 3D workload at its full 64^3 macro grid: one box near the centre
CASES["c4_3d_full"] = ("c4_3d", {}, [32 * 64 * 64 + 32 * 64 + 32])


def _one(item):
    import numpy as np
    import workloads as W
    from oracle import hmm_oracle as O
    name, (wl, over, pts) = item
    cfg = W.config(wl, **over)
    M0 = W.initial_field(cfg)
    H = O.micro_batch(cfg, M0, points=pts, dtype=np.longdouble)
    return name, dict(workload=wl, overrides=over, points=pts,
                      H=[[float(H[c, i]) for i in range(len(pts))] for c in range(3)])


def main():
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        res = dict(pool.map(_one, sorted(CASES.items())))
    import numpy as np
    rec = {"generator": "tests/golden/make_longdouble_refs.py",
           "arithmetic": f"numpy longdouble ({np.finfo(np.longdouble).nmant + 1}-bit significand) on {platform.machine()}",
           "cases": res}
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
    print(OUT)


if __name__ == "__main__":
    main()
