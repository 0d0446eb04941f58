#!/usr/bin/env python3
"""Benchmark of the HMM micro-problem path on GB300.

The headline workload is the field model's HMM (MPEA macro steps, Section 3.1)
on the 3D workload at its full size: a 64^3 periodic macro grid, one 32^3-node
micro box per macro point (262,144 micro problems), 300 HeunP micro steps each,
eps = 1/100, a = 1 + 0.5 sin(2 pi y1) sin(2 pi y2) sin(2 pi y3), alpha = 0.1,
alpha_micro = 1.2, 4th-order stencil: 1.38e12 lattice updates per macro step.
Each macro step is taken in 16 waves (hmm_macro_step_wave), and a benchmark
step is one wave: the micro batch of 16,384 of the boxes (8.6e10 lattice
updates), the wave that ends a macro step adding the MPEA update of every
point. The headline value is micro lattice updates per second of the batched FP32 form;
the plain FP64 method is timed on a sample of the same boxes. The line carries
the same measurements for the uneven 2D workload (256^2 macro grid, boxes of
32^2 to 96^2) and the 128^2 2D workload as sub-objects.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The line also carries a "dns" object: the direct simulation resolving eps
(Section 5's reference solver) on the paper's quasi-periodic 2D grid (1500^2),
point-steps/s of the float-float FP32 form against the measured HBM bandwidth,
and the FP64 form beside it (--no-dns leaves it out; --dns prints it alone).

Multi-GPU: each rank runs an independent replica (the micro problems of one
macro grid are independent; no collective on the data path), the value is
the total over ranks divided by the slowest rank's time (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "micro lattice updates/s + HMM macro steps/s, FP32-batched vs FP64, <=1e-6 rel err"
UNIT = "LU/s"
WORKLOAD = "c4_3d"
# Algorithmic FP32 flops per lattice update of HeunP with the order-4 staggered stencil
# (no compensation terms): per stage the stencil costs 9 flops per axis and component
# (one face flux of 5, one node combination of 4) plus 2 for H = cs Hs + H(m_init) per
# component, the right-hand side 27 (m = m_init + v, two cross products, the damping
# fma); the stages' combination, projection and update 42; the average 6. 2D: 2 x 60 +
# 54 + 42 + 6 = 222; 3D: 2 x 87 + 54 + 42 + 6 = 276.
FLOPS_PER_LU = {2: 222.0, 3: 276.0}
BYTES_PER_LU_FP32 = 24.0    # streaming-model bytes per lattice update: 3-component FP32 state read and written
FP32_LANES_PER_SM = 128
WORKLOADS = {
    "c4_3d": dict(
        desc=("3D HMM, 64^3 periodic macro grid, 262144 micro boxes of 32^3 nodes (6 per eps, eps=1/100), "
              "300 HeunP micro steps, 4th-order stencil, a=1+0.5 sin(2pi y1)sin(2pi y2)sin(2pi y3), "
              "alpha=0.1, alpha_micro=1.2"),
        kernel="micro_fp32_3d_col_kernel<3> (z-column, shared-memory resident, 9-CTA clusters)",
        traffic="micro_fp32_3d_col_c4_traffic.txt", source="micro_fp32_3d_col.cuh",
        steps=16, waves=16, e2e_steps=1, fp64_sample=4096),
    "c3_2d_uneven": dict(
        desc=("2D HMM, 256^2 macro grid, 65536 uneven micro boxes of 32^2 to 96^2 nodes (eps_i in "
              "[1/400, 1/100], 8 per eps_i), 400 HeunP micro steps, a=1.1+0.25sin(2pi y1)cos(2pi y2)"
              "+0.25sin(2pi x1)sin(2pi y2), alpha=0.01, alpha_micro=1.2"),
        kernel="micro_fp32_2d_kernel instances (shared-memory resident; packs and clusters)",
        traffic=None, source="micro_fp32_2d.cuh", steps=3, e2e_steps=2, fp64_sample=1024),
    "c2_2d": dict(
        desc=("2D HMM, 128^2 periodic macro grid, 16384 micro boxes of 64^2 nodes (8 per eps, eps=1/200), "
              "400 HeunP micro steps, 4th-order stencil, a=1+0.5sin(2pi y1)sin(2pi y2), alpha=0.05, "
              "alpha_micro=1.2"),
        kernel="micro_fp32_2d_kernel<3,4,64,58> (shared-memory resident)",
        traffic="micro_fp32_2d_c2_traffic.txt", source="micro_fp32_2d.cuh", steps=10, e2e_steps=5,
        fp64_sample=4096),
}
SUB_WORKLOADS = ("c3_2d_uneven", "c2_2d")


DNS_TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dns_kernel_quasi2d_traffic.txt")
DNS_KERNEL_SOURCE = os.path.join(ROOT, "paper_2108_09463_gb300", "csrc", "dns_kernels.cuh")


def _traffic_from_profile(traffic_file, kernel_source):
    """ncu DRAM bytes per full launch recorded for this kernel source, else None.

    The profile summary carries the SHA-256 of the kernel source it was captured
    from; once the source changes the figure no longer applies and None is returned.
    """
    if not traffic_file:
        return None
    try:
        kv = dict(line.split(":", 1) for line in open(traffic_file) if ":" in line)
        sha = hashlib.sha256(open(kernel_source, "rb").read()).hexdigest()
        if kv["kernel_source_sha256"].strip() != sha:
            return None
        return float(kv["dram_bytes_per_full_launch"])
    except (OSError, KeyError, ValueError):
        return None


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------- CPU oracle leg
_INPUTS = {}   # per worker process: the workload's seeded macro field, generated once


def _oracle_chunk(args):
    """The oracle on a list of boxes in one worker; returns (worker pid, seconds of
    the solve alone: the input generation is not timed)."""
    name, over, points = args
    import workloads as W
    from oracle import hmm_oracle as O
    cfg = W.config(name, **over)
    key = (name, tuple(sorted(over.items())))
    if key not in _INPUTS:
        _INPUTS[key] = W.initial_field(cfg)
    M0 = _INPUTS[key]
    t = time.perf_counter()
    if getattr(cfg, "model", 0) == 1:
        from oracle import flux_oracle as F
        F.micro_batch_flux(cfg, M0, points=points)
    else:
        O.micro_batch(cfg, M0, points=points)
    return os.getpid(), time.perf_counter() - t


def oracle_sample(name: str, boxes_per_worker: int, workers: int, pool=None, over=None):
    """Time the oracle on a bounded sample of boxes of the workload; returns (LU/s, info).

    The boxes are spread over the grid, boxes_per_worker per worker process; the
    time is the longest total solve time of any worker (the workers run at once)."""
    import workloads as W
    from oracle import hmm_oracle as O
    over = dict(over or {})
    cfg = W.config(name, **over)
    n = workers * boxes_per_worker
    stride = max(1, cfg.n_points // n)
    pts = [i * stride for i in range(n)]
    chunks = [(name, over, pts[w * boxes_per_worker:(w + 1) * boxes_per_worker]) for w in range(workers)]
    if pool is None:
        res = [_oracle_chunk(c) for c in chunks]
    else:
        res = pool.map(_oracle_chunk, chunks, chunksize=1)
    per_worker = {}
    for pid, t in res:
        per_worker[pid] = per_worker.get(pid, 0.0) + t
    wall = max(per_worker.values())
    lu = 0.0
    boxes_per_point = cfg.dim if getattr(cfg, "model", 0) == 1 else 1   # the flux model: one box per axis
    for p in pts:
        g = O.box_geometry(cfg, p)
        lu += boxes_per_point * (g["N"] - 2 * g["r"]) ** cfg.dim * g["M"]
    return lu / wall, dict(boxes=n, wall_s=wall, lu=lu, workers_used=len(per_worker))


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # the raw samples: HMM_BENCH_CLOCKS_DIR if set, else the system's temporary directory
        out_dir = os.environ.get("HMM_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- our arm
def aggregate_ranks(ms_local: float, world: int, steps: int, units_per_step: float, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas (weak scaling): the slowest
    rank's time (max over ranks, the only collective, outside the data path)
    and units = world x steps x units_per_step over it. Returns (ms_max, value)."""
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * steps * units_per_step / (ms_max / 1e3)


def _timed(fn, k, flush):
    """k calls of fn, each bracketed by CUDA events on the current stream, L2 flushed
    between them (a write larger than L2); returns the total device ms."""
    import torch
    tot = 0.0
    for _ in range(k):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    return tot


def fp32_rates():
    """Measured FP32 FMA rates of this GPU in TFLOP/s (scalar and paired FP32x2 FMAs)."""
    from paper_2108_09463_gb300 import fp32_fma_rate
    return {"scalar": fp32_fma_rate(packed=False) / 1e12, "packed": fp32_fma_rate(packed=True) / 1e12}


def measure_workload(name, steps, warmup, flush, world=1, dist=None, pool=None, cpu_workers=16,
                     cpu_boxes_per_worker=1, kernel_reps=2, fma=None):
    """The batched FP32 form on one workload: `warmup` then `steps` MPEA macro steps
    (value = lattice updates/s over the timed steps), the dominant kernel's time per
    launch from the library's events on its stream, the roofline, end to end through
    the host-buffer entry point, the FP64 method on a sample of the same boxes, and
    the oracle on a bounded sample of boxes (spawned processes on the host cores).

    A workload with `waves` > 1 takes each macro step in that many calls of
    hmm_macro_step_wave (one step = one wave: the micro batch of 1/waves of the
    boxes; the wave that ends a macro step adds the MPEA update of every point),
    and the dominant kernel's time is the mean of the timed waves' micro batches."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2108_09463_gb300 import HMM
    spec = WORKLOADS[name]
    cfg = W.config(name)
    M0 = W.initial_field(cfg)
    h32 = HMM(cfg, precision=1)
    lu_batch, _ = h32.stats()
    plan = h32.plan_report().strip()
    # MPEA steps from a restart state (history zero, j = 2): every step is a full micro
    # batch and an MPEA update; the RK4P start-up (4 micro batches a step) is not timed
    hist = torch.zeros((2, 3, cfg.n_points), dtype=torch.float64, device="cuda")
    h32.set_state(hist, 2)
    M = torch.from_numpy(M0).cuda()
    nw = spec.get("waves", 1)
    if nw > 1:
        # every wave holds the same number of equal boxes, so a step is lu_batch / nw
        assert cfg.box_n_field is None and cfg.eps_field is None and cfg.n_points % nw == 0
    lu_step = lu_batch / nw
    wave = [0, 0, []]    # next wave, macro steps completed in the timed region, wave kernel ms

    def one_step(timed):
        if nw == 1:
            h32.macro_step(M, 1)
            return
        h32.macro_step_wave(M, wave[0], nw)
        if timed:
            wave[2].append(h32.stats()[1])
            wave[1] += wave[0] == nw - 1
        wave[0] = (wave[0] + 1) % nw

    for _ in range(warmup):
        one_step(False)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    with ClockSampler(torch.cuda.current_device()) as clk:
        ms = _timed(lambda: one_step(True), steps, flush)
    torch.cuda.synchronize()
    ms_max, value = aggregate_ranks(ms, world, steps, lu_step, dist, "cuda")
    if nw > 1:
        # the dominant kernel: the timed waves' micro batches, each timed on the
        # library's stream by its own events
        k_ms = sum(wave[2]) / len(wave[2])
        launches = steps * sum(1 for ln in plan.splitlines() if ln.startswith("3D")) + 2 * wave[1]
    else:
        # the dominant kernel: one micro batch, timed per launch on the library's stream
        H = torch.empty_like(M)
        kms = []
        # (one launch when a step takes more than 10 s: its time is already a long average)
        for _ in range(kernel_reps if ms / steps < 1e4 else 1):
            flush.zero_()
            h32.micro_batch(M, H)
            kms.append(h32.stats()[1])
        k_ms = min(kms)
        launches = 3 * steps
    peaks = _peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    derived = n_sm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    # the denominator: the larger of the lanes-times-clock figure and the measured rate of
    # the paired FP32x2 FMAs the kernels issue, so that the fraction is never flattered
    alu_peak = max(derived, fma["packed"]) if fma else derived
    flops = FLOPS_PER_LU[cfg.dim] * lu_step
    achieved = flops / (k_ms / 1e3) / 1e12
    hbm = peaks.get("hbm_gbs", 6800.0)
    traffic = None
    if spec["traffic"]:
        traffic = _traffic_from_profile(os.path.join(ROOT, "profiles", spec["traffic"]),
                                        os.path.join(ROOT, "paper_2108_09463_gb300", "csrc", spec["source"]))
        if traffic is not None:
            traffic /= nw   # recorded per launch over every box; a wave's launch holds 1/nw of them
    stream_gbs = BYTES_PER_LU_FP32 * lu_step / (k_ms / 1e3) / 1e9
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "traffic": traffic, "kernel": spec["kernel"], "kernel_ms": k_ms,
                "flops_per_lu": FLOPS_PER_LU[cfg.dim],
                "peak_source": (f"max of the FP32 FMA lanes x clock ({n_sm} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x "
                                f"{sm_max:.0f} MHz = {derived:.1f} TFLOP/s) and the FMA rate measured by "
                                "hmm_fp32_fma_rate on this GPU (no FP32 figure in MEASURED_PEAKS.json)"),
                "peak_derived": derived,
                "fp32_fma_measured_tflops": fma,
                "hbm_streaming_equivalent": {"GB_per_s": stream_gbs, "frac_of_measured_hbm": stream_gbs / hbm,
                                             "bytes_per_lu": BYTES_PER_LU_FP32}}
    # end to end through hmm_macro_step_host: pinned host M in and out every step
    Mh = M.cpu().pin_memory()
    ke = spec["e2e_steps"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        h32.macro_step_host(Mh.numpy(), 1)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * ke * lu_batch / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": 3 * cfg.n_points * 8, "d2h_bytes_per_step": 3 * cfg.n_points * 8,
           "macro_steps_per_s": ke / e2e_s, "steps": ke, "entry_point": "hmm_macro_step_host"}
    # the plain FP64 method: the whole batch, or a spread sample of its boxes through
    # hmm_micro_batch_points when the whole batch would take minutes
    h64 = HMM(cfg, precision=0)
    nsamp = spec["fp64_sample"]
    Mfix = torch.from_numpy(M0).cuda()
    H32 = h32.micro_batch(Mfix).cpu().numpy()
    info = h32.box_info()
    if nsamp:
        pts = np.linspace(0, cfg.n_points - 1, nsamp).astype(np.int64)
        pts = np.unique(pts)
        h64.micro_batch_points(Mfix, pts[:64])      # warm-up (allocates the subset tables)
        H64f = h64.micro_batch_points(Mfix, pts).cpu().numpy()
        ms64 = h64.stats()[1]
        lu64_batch = float(np.sum((info["N"][pts] - 6.0) ** cfg.dim) * cfg.micro_steps)
        sel = pts
        fp64_desc = f"hmm_micro_batch_points on {len(pts)} boxes spread over the grid"
    else:
        H64f = h64.micro_batch(Mfix).cpu().numpy()
        ms64 = h64.stats()[1]
        lu64_batch = lu_batch
        sel = slice(None)
        fp64_desc = "hmm_micro_batch on the whole batch"
    lu64 = lu64_batch / (ms64 / 1e3)
    rel = float(np.linalg.norm(H32[:, sel] - H64f[:, sel], axis=0).max() / np.linalg.norm(H64f[:, sel], axis=0).max())
    h64.close()
    h32.close()
    out = {"workload": spec["desc"], "name": name, "value": value, "unit": UNIT, "steps": steps, "warmup": warmup,
           "ms_per_step": ms_max / steps, "macro_steps_per_s": steps / nw / (ms_max / 1e3), "lu_per_step": lu_step,
           "waves_per_macro_step": nw, "lu_per_macro_step": lu_batch,
           "boxes": cfg.n_points, "micro_steps": cfg.micro_steps,
           "fp64_plain": {"value": lu64, "unit": UNIT, "how": fp64_desc, "kernel_ms": ms64},
           "speedup_fp32_vs_fp64": value / world / lu64,
           "fp32_vs_fp64_rel_err": rel,
           "roofline": roofline, "e2e": e2e, "plan": plan,
           "gpu_launches": launches, "clocks": clk.summary()}
    if pool is not None:
        oracle_sample(name, 1, cpu_workers, pool)   # each worker generates the seeded input once, untimed
        v, sinfo = oracle_sample(name, cpu_boxes_per_worker, cpu_workers, pool)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": sinfo["workers_used"], "kind": "oracle",
                               "sample": f"{sinfo['boxes']} of the {cfg.n_points} micro boxes (whole boxes, all "
                                         f"{cfg.micro_steps} micro steps), {cpu_workers} spawned processes, "
                                         f"{sinfo['wall_s']:.1f} s for the slowest worker's solves"}
    else:
        out["cpu_baseline"] = None
    return out


CPU_BOXES = {"c4_3d": 4, "c3_2d_uneven": 4, "c2_2d": 16}


def _warm_worker(_):
    import workloads  # noqa: F401
    from oracle import hmm_oracle  # noqa: F401
    return 0


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2108_09463_gb300 import build

    # Spawned CPU workers for the oracle baseline start before any GPU work.
    pool = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = mp.get_context("spawn").Pool(args.cpu_workers)

    build()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    if pool is not None:
        pool.map(_warm_worker, range(args.cpu_workers))   # imports, outside every timed sample
    steps = args.steps if args.steps is not None else WORKLOADS[args.headline]["steps"]
    fma = fp32_rates()
    head = measure_workload(args.headline, steps, args.warmup, flush, world, dist, pool, args.cpu_workers,
                            CPU_BOXES.get(args.headline, 2), args.kernel_reps, fma)
    clocks = head["clocks"]
    subs = {}
    if not args.no_sub:
        for name in SUB_WORKLOADS:
            if name == args.headline:
                continue
            subs[name] = measure_workload(name, WORKLOADS[name]["steps"], max(3, args.warmup), flush, world, dist,
                                          pool, args.cpu_workers, CPU_BOXES.get(name, 4), args.kernel_reps, fma)
    if pool is not None:
        pool.close()

    dns = None
    if rank == 0 and not args.no_dns:
        # the direct simulation resolving eps (Section 5's reference solver) on the
        # paper's quasi-periodic 2D grid: float-float FP32 form and FP64 form
        r32 = dns_measure(DNS_WORKLOAD, "fp32", 2004, 50)
        r64 = dns_measure(DNS_WORKLOAD, "fp64", 204, 50)
        hbm = _peaks().get("hbm_gbs", 6800.0)
        dns = {k: r32[k] for k in ("workload", "grid", "value", "unit", "ms_per_step", "steps", "dt",
                                   "bytes_per_point_step", "achieved_gbs", "achieved_gbs_without_coefficient")}
        dns["roofline"] = {"bound": "hbm", "achieved": r32["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                           "frac": r32["achieved_gbs"] / hbm,
                           "traffic": _traffic_from_profile(DNS_TRAFFIC_FILE, DNS_KERNEL_SOURCE)}
        dns["fp64"] = {"value": r64["value"], "ms_per_step": r64["ms_per_step"], "steps": r64["steps"]}
        dns["speedup_vs_fp64"] = r32["value"] / r64["value"]
        if not args.no_cpu_baseline:
            v, sample = dns_oracle_sample()
            dns["cpu_baseline"] = {"value": v, "unit": "point-steps/s", "cores": 1, "kind": "oracle", "sample": sample}

    if rank == 0:
        spec = WORKLOADS[args.headline]
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": spec["desc"], "name": args.headline, "boxes": head["boxes"],
                       "micro_steps": head["micro_steps"], "lu_per_step": head["lu_per_step"],
                       "precision": "fp32-batched",
                       "step": ("one MPEA macro step (one micro batch over every box + the MPEA update), "
                                "from a restart state" if head["waves_per_macro_step"] == 1 else
                                f"one wave of an MPEA macro step taken in {head['waves_per_macro_step']} waves "
                                f"(hmm_macro_step_wave): the micro batch of {head['boxes'] // head['waves_per_macro_step']} "
                                f"of the {head['boxes']} boxes; every {head['waves_per_macro_step']}th wave ends the "
                                "macro step with the MPEA update of every point; from a restart state"),
                       "lu_per_macro_step": head["lu_per_macro_step"],
                       "l2": "flushed (256 MB write) between timed steps; the working set is larger than L2",
                       "parallelism": f"replicas x{world}"},
            "macro_steps_per_s": head["macro_steps_per_s"],
            "fp64_plain": head["fp64_plain"],
            "speedup_fp32_vs_fp64": head["speedup_fp32_vs_fp64"],
            "fp32_vs_fp64_rel_err": head["fp32_vs_fp64_rel_err"],
            "roofline": head["roofline"], "cpu_baseline": head["cpu_baseline"], "e2e": head["e2e"],
            "clocks": clocks,
            "gpu_launches": head["gpu_launches"],
            "plan": head["plan"],
            "workloads": subs,
            "dns": dns,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------- micro-batch mode
def run_micro_only(args, local_rank):
    """Time hmm_micro_batch alone (the hot path) on a workload of any grid size.

    Prints one JSON line per run: LU/s and the per-launch device time from the
    library's events on its launch stream.
    """
    import torch
    import workloads as W
    from paper_2108_09463_gb300 import HMM, build
    build()
    torch.cuda.set_device(local_rank)
    over = {}
    if args.macro_grid:
        n = list(args.macro_grid) + [1] * (3 - len(args.macro_grid))
        over["n_macro"] = tuple(n)
    if args.box_n:
        over["box_n"] = args.box_n
    if args.alpha_micro:
        over["alpha_micro"] = args.alpha_micro
    if args.micro_stepper:
        over["micro_stepper"] = args.micro_stepper
    if args.model:
        over["model"] = args.model
    cfg = W.config(args.workload, **over)
    if args.workload == "c3_2d_uneven" and args.macro_grid:
        cfg = cfg.replace(eps_field=None, box_n_field=None)
        eps, nf = W.uneven_eps_and_n(cfg)
        cfg = cfg.replace(eps_field=eps, box_n_field=nf)
    prec = 0 if args.precision == "fp64" else 1
    table = W.face_table(cfg) if cfg.coef_fn is not None else None
    h = HMM(cfg, precision=prec, kernel_variant=args.variant, face_table=table)
    M = torch.from_numpy(W.initial_field(cfg)).cuda()
    H = torch.empty_like(M)
    for _ in range(args.warmup):
        h.micro_batch(M, H)
    ms = []
    for _ in range(args.steps):
        h.micro_batch(M, H)
        ms.append(h.stats()[1])
    lu = h.stats()[0]
    rec = {"mode": "micro-only", "workload": args.workload, "boxes": cfg.n_points,
           "precision": args.precision, "variant": args.variant, "lu_per_batch": lu,
           "ms_per_batch": sum(ms) / len(ms), "LU_per_s": lu / (sum(ms) / len(ms) / 1e3), "ms": ms,
           "micro_stepper": ["HeunP", "RK4P", "MPE", "MPEA"][cfg.micro_stepper], "model": ["field", "flux"][cfg.model],
           "micro_dt_mean": float(h.box_info()["dt"].mean()), "micro_steps": cfg.micro_steps,
           "plan": h.plan_report().strip(), "fp32_fma_measured_tflops": fp32_rates()}
    if args.cpu_baseline_micro:
        # the oracle on a spread sample of the same boxes, spawned processes on the host cores
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(args.cpu_workers) as pool:
            oracle_sample(args.workload, 1, args.cpu_workers, pool, over)   # warm the workers
            v, info = oracle_sample(args.workload, args.cpu_boxes_per_worker, args.cpu_workers, pool, over)
        rec["cpu_baseline"] = {"value": v, "unit": "LU/s", "cores": args.cpu_workers, "kind": "oracle",
                               "sample": f"{info['boxes']} of the {cfg.n_points} boxes, {info['wall_s']:.1f} s wall"}
    if args.macro_steps > 0:
        # steady-state macro steps (MPEA, one micro batch each, graph replay) after
        # the RK4P start-up steps j = 0, 1 and one warm-up step
        # (--waves n: each timed macro step in n calls of hmm_macro_step_wave)
        h.macro_step(M, 3)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        if args.waves > 1:
            for _ in range(args.macro_steps):
                for w in range(args.waves):
                    h.macro_step_wave(M, w, args.waves)
        else:
            h.macro_step(M, args.macro_steps)
        t1.record()
        torch.cuda.synchronize()
        sec = t0.elapsed_time(t1) / 1e3
        rec.update(macro_steps=args.macro_steps, macro_steps_per_s=args.macro_steps / sec, waves=args.waves)
    h.close()
    print(json.dumps(rec), flush=True)


# ---------------------------------------------------------------- direct simulation
DNS_WORKLOAD = "dns_quasi2d"
# Bytes one time step must move per grid point: state read and write,
# two history reads and one write, and the two face coefficients. float-float
# form: 24 + 24 + 24 + 12 + 8 = 92; FP64: 24 + 24 + 48 + 24 + 16 = 136. (Without
# the coefficient reads, which a separable coefficient could avoid, 84 and 120.)
DNS_BYTES_PER_PT = {"fp32": 92.0, "fp64": 136.0}


def dns_measure(workload=DNS_WORKLOAD, precision="fp32", steps=1000, warmup=50, grid=None):
    """Time hmm_dns_step on a named direct simulation: ``warmup`` steps (the
    RK4P start-up and the first MPEA steps), then ``steps`` MPEA steps in one
    call, timed by the library's events on its stream. Inputs are resident in
    HBM; the per-step working set (state, history) is larger than L2 at 1500^2
    (189 MB in the float-float form). Returns a dict."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2108_09463_gb300 import DNS
    over = {}
    if grid:
        over["n"] = tuple(list(grid) + [1] * (3 - len(grid)))
    cfg = W.dns_config(workload, **over)
    prec = 0 if precision == "fp64" else 1
    table = None
    if cfg.coef_fn is not None:
        X = W.dns_coords(cfg)
        dxs = [cfg.L / n for n in cfg.shape]
        blocks = []
        for k in range(cfg.dim):
            P = np.meshgrid(*[x + (0.5 * dxs[a] if a == k else 0.0) for a, x in enumerate(X)], indexing="ij")
            blocks.append(np.asarray(cfg.coef_fn(P, cfg.eps), dtype=np.float64).ravel())
        table = np.concatenate(blocks)
    d = DNS(cfg, precision=prec, face_table=table)
    M = torch.from_numpy(W.dns_initial(cfg)).cuda()
    d.step(M, warmup)
    d.step(M, steps)
    ms = d.info()["last_ms"]
    info = d.info()
    d.close()
    G = cfg.n_points
    ms_step = ms / steps
    return {"workload": workload, "grid": list(cfg.shape), "precision": precision, "steps": steps,
            "ms_per_step": ms_step, "value": G / (ms_step / 1e3), "unit": "point-steps/s",
            "dt": info["dt"], "bytes_per_point_step": DNS_BYTES_PER_PT[precision],
            "achieved_gbs": DNS_BYTES_PER_PT[precision] * G / (ms_step / 1e3) / 1e9,
            "achieved_gbs_without_coefficient": (DNS_BYTES_PER_PT[precision] - (8.0 if precision == "fp32" else 16.0))
            * G / (ms_step / 1e3) / 1e9,
            "finite": bool(torch.isfinite(M).all())}


def dns_oracle_sample(workload=DNS_WORKLOAD, n=150, steps=8):
    """Time the direct-simulation oracle on an n x n (n for 1D) grid of the same
    coefficient and spacing scale, `steps` steps (the RK4P start-up included);
    returns (point-steps/s, sample description). Single process (numpy)."""
    import workloads as W
    from oracle import dns_oracle as D
    cfg = W.dns_config(workload)
    cfg = cfg.replace(n=tuple([n] * cfg.dim + [1] * (3 - cfg.dim)))
    M0 = W.dns_initial(cfg)
    run = D.DNS(cfg, M0)
    t = time.perf_counter()
    run.step(steps)
    wall = time.perf_counter() - t
    return cfg.n_points * steps / wall, (f"{'x'.join(map(str, cfg.shape))} grid of {workload}'s coefficient, "
                                         f"{steps} steps (2 RK4P + {steps - 2} MPEA), 1 process, {wall:.1f} s wall")


def run_dns(args, local_rank):
    """--dns: one JSON line for the direct simulation (float-float FP32 form and
    the FP64 form on the same grid)."""
    import torch
    from paper_2108_09463_gb300 import build
    build()
    torch.cuda.set_device(local_rank)
    wl = args.workload if args.workload.startswith("dns_") else DNS_WORKLOAD
    rec = {"mode": "dns"}
    with ClockSampler(local_rank) as clk:
        r32 = dns_measure(wl, "fp32", args.steps, args.warmup, args.macro_grid)
        r64 = dns_measure(wl, "fp64", max(1, args.fp64_steps), args.warmup, args.macro_grid) if args.fp64_steps > 0 else None
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    rec.update(r32)
    traffic = _traffic_from_profile(DNS_TRAFFIC_FILE, DNS_KERNEL_SOURCE) if wl == DNS_WORKLOAD and not args.macro_grid else None
    rec["roofline"] = {"bound": "hbm", "achieved": r32["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                       "frac": r32["achieved_gbs"] / hbm, "traffic": traffic,
                       "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback 6800 GB/s"}
    if r64:
        rec["fp64"] = r64
        rec["speedup_vs_fp64"] = r32["value"] / r64["value"]
    rec["clocks"] = clk.summary()
    if not args.no_cpu_baseline:
        v, sample = dns_oracle_sample(wl)
        rec["cpu_baseline"] = {"value": v, "unit": "point-steps/s", "cores": 1, "kind": "oracle", "sample": sample}
    print(json.dumps(rec), flush=True)


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    workers = args.cpu_workers
    pool = mp.get_context("spawn").Pool(workers)
    pool.map(_warm_worker, range(workers))
    name = args.headline
    steps = args.steps if args.steps is not None else WORKLOADS[name]["steps"]
    for _ in range(args.warmup):
        oracle_sample(name, 1, workers, pool)
    tot_lu, tot_s = 0.0, 0.0
    for _ in range(steps):
        v, info = oracle_sample(name, args.ref_boxes_per_worker, workers, pool)
        tot_lu += info["lu"]
        tot_s += info["wall_s"]
    pool.close()
    value = tot_lu / tot_s
    import workloads as W
    cfg = W.config(name)
    sample = (f"each step: {workers * args.ref_boxes_per_worker} of the {cfg.n_points} micro boxes "
              f"(whole boxes, all {cfg.micro_steps} micro steps), {workers} spawned processes")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOADS[name]["desc"], "name": name,
                                        "precision": "fp64 oracle",
                                        "step": f"a bounded sample of the workload: {workers * args.ref_boxes_per_worker} "
                                                "whole micro boxes (all micro steps), one per worker"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps of the headline workload (default: 16 for the 3D workload, whose step "
                         "is one of the 16 waves of a macro step)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--kernel-reps", type=int, default=2)
    ap.add_argument("--cpu-workers", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--cpu-boxes-per-worker", type=int, default=16)
    ap.add_argument("--ref-boxes-per-worker", type=int, default=1)
    ap.add_argument("--headline", default=WORKLOAD, choices=sorted(WORKLOADS),
                    help="workload of the headline value (the others become sub-objects)")
    ap.add_argument("--no-sub", action="store_true", help="leave the other workloads' sub-objects out")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--micro-only", action="store_true",
                    help="time hmm_micro_batch alone (see --workload, --macro-grid, --precision, --variant)")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--macro-grid", type=int, nargs="+", default=None)
    ap.add_argument("--box-n", type=int, default=None)
    ap.add_argument("--alpha-micro", type=float, default=None)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--variant", type=int, default=0, help="FP32 kernel: 0 automatic, 1 generic, 2 resident")
    ap.add_argument("--micro-stepper", type=int, default=0, choices=[0, 1, 2, 3],
                    help="with --micro-only: 0 HeunP, 1 RK4P, 2 MPE, 3 MPEA")
    ap.add_argument("--model", type=int, default=0, help="with --micro-only: 0 field model, 1 flux model (FP64)")
    ap.add_argument("--cpu-baseline-micro", action="store_true",
                    help="with --micro-only: also time the oracle on a sample of the boxes")
    ap.add_argument("--no-dns", action="store_true",
                    help="leave the direct-simulation measurement out of the default line")
    ap.add_argument("--dns", action="store_true",
                    help="time the direct simulation (--workload dns_*, --macro-grid for its grid, "
                         "--steps MPEA steps, --fp64-steps for the FP64 form)")
    ap.add_argument("--waves", type=int, default=1,
                    help="with --micro-only --macro-steps: take each timed macro step in this many waves")
    ap.add_argument("--macro-steps", type=int, default=0,
                    help="with --micro-only: also time this many steady-state macro steps")
    args = ap.parse_args()
    if args.steps is None and (args.micro_only or args.dns):
        args.steps = 10
    if args.warmup < 3 and not (args.micro_only or args.dns):
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.dns:
        run_dns(args, local_rank)
    elif args.micro_only:
        run_micro_only(args, local_rank)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
