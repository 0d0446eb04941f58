#!/usr/bin/env python3
"""Benchmark of the HMM micro-problem path on GB300.

A step is one full HMM macro step (MPEA, Section 3.1) of the field model on the
2D workload: a 128^2 periodic macro grid, one 64^2-node micro box per macro
point (16384 micro problems), 400 HeunP micro steps each, eps = 1/200,
a = 1 + 0.5 sin(2 pi y1) sin(2 pi y2), alpha = 0.05, alpha_micro = 1.2,
4th-order stencil. The headline value is micro lattice updates per second of
the batched FP32 form; the plain FP64 method is timed on the same workload.

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
WORKLOAD = "c2_2d"
WORKLOAD_DESC = ("2D HMM, 128^2 periodic macro grid, 16384 micro boxes of 64^2 nodes "
                 "(8 per eps, eps=1/200), 400 HeunP micro steps, 4th-order stencil, "
                 "a=1+0.5sin(2pi y1)sin(2pi y2), alpha=0.05, alpha_micro=1.2")
FLOPS_PER_LU_2D = 255.0     # algorithmic FP32 flops per lattice update, 2D order 4: stencil 120,
                            # m = m_init + v 6, right-hand side 48, stage 1 18, stage 2 63
BYTES_PER_LU_FP32 = 24.0    # streaming-model bytes per lattice update: 3-component FP32 state read and written
FP32_LANES_PER_SM = 128


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "micro_fp32_2d_c2_traffic.txt")
KERNEL_SOURCE = os.path.join(ROOT, "paper_2108_09463_gb300", "csrc", "micro_fp32_2d.cuh")
DNS_TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dns_kernel_quasi2d_traffic.txt")
DNS_KERNEL_SOURCE = os.path.join(ROOT, "paper_2108_09463_gb300", "csrc", "dns_kernels.cuh")


def _traffic_from_profile(traffic_file=None, kernel_source=None):
    """ncu DRAM bytes per full launch recorded for this kernel source, else None.

    The profile summary carries the SHA-256 of the kernel source it was captured
    from; once the source changes the figure no longer applies and None is returned.
    """
    try:
        kv = dict(line.split(":", 1) for line in open(traffic_file or TRAFFIC_FILE) if ":" in line)
        sha = hashlib.sha256(open(kernel_source or KERNEL_SOURCE, "rb").read()).hexdigest()
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
def _oracle_chunk(args):
    name, over, points = args
    import workloads as W
    from oracle import hmm_oracle as O
    cfg = W.config(name, **over)
    M0 = W.initial_field(cfg)
    t = time.perf_counter()
    if getattr(cfg, "model", 0) == 1:
        from oracle import flux_oracle as F
        F.micro_batch_flux(cfg, M0, points=points)
    else:
        O.micro_batch(cfg, M0, points=points)
    return time.perf_counter() - t


def oracle_sample(name: str, boxes_per_worker: int, workers: int, pool=None, over=None):
    """Time the oracle on a bounded sample of boxes of the workload; returns (LU/s, info)."""
    import workloads as W
    from oracle import hmm_oracle as O
    over = dict(over or {})
    cfg = W.config(name, **over)
    n = workers * boxes_per_worker
    stride = max(1, cfg.n_points // n)
    pts = [i * stride for i in range(n)]
    chunks = [(name, over, pts[w * boxes_per_worker:(w + 1) * boxes_per_worker]) for w in range(workers)]
    t0 = time.perf_counter()
    if pool is None:
        for c in chunks:
            _oracle_chunk(c)
    else:
        pool.map(_oracle_chunk, chunks)
    wall = time.perf_counter() - t0
    lu = 0.0
    boxes_per_point = cfg.dim if getattr(cfg, "model", 0) == 1 else 1   # the flux model: one box per axis
    for p in pts:
        g = O.box_geometry(cfg, p)
        lu += boxes_per_point * (g["N"] - 2 * g["r"]) ** cfg.dim * g["M"]
    return lu / wall, dict(boxes=n, wall_s=wall, lu=lu)


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


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import workloads as W
    from paper_2108_09463_gb300 import HMM, build

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

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    cfg = W.config(WORKLOAD)
    M0 = W.initial_field(cfg)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def timed_steps(fn, k):
        """k calls of fn, each bracketed by CUDA events on the current stream, L2 flushed between."""
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

    # --- FP32 batched form: full macro steps (RK4P start-up inside warm-up, then MPEA).
    h32 = HMM(cfg, precision=1)
    lu_batch, _ = h32.stats()
    plan = h32.plan_report().strip()   # the resident-plan autotuner's timings at init
    M = torch.from_numpy(M0).cuda()
    for _ in range(args.warmup):
        h32.macro_step(M, 1)
    barrier()
    with ClockSampler(local_rank) as clk:
        ms32 = timed_steps(lambda: h32.macro_step(M, 1), args.steps)
    barrier()
    ms_max, value = aggregate_ranks(ms32, world, args.steps, lu_batch, dist, "cuda")
    macro_steps_per_s = args.steps / (ms_max / 1e3)

    # --- dominant kernel: the FP32 micro-batch kernel, timed per launch on its stream.
    H = torch.empty_like(M)
    kms = []
    for _ in range(args.kernel_reps):
        flush.zero_()
        h32.micro_batch(M, H)
        kms.append(h32.stats()[1])
    k_ms = sum(kms) / len(kms)
    flops = FLOPS_PER_LU_2D * lu_batch
    peaks = _peaks()
    clocks = clk.summary()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    props = torch.cuda.get_device_properties(local_rank)
    n_sm = props.multi_processor_count
    alu_peak = n_sm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = flops / (k_ms / 1e3) / 1e12
    hbm = peaks.get("hbm_gbs", 6800.0)
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak,
                "traffic": args.traffic if args.traffic is not None else _traffic_from_profile(),
                "kernel": "micro_fp32_2d_kernel<3,4,64,58> (shared-memory resident)", "kernel_ms": k_ms,
                "peak_source": f"FP32 FMA: {n_sm} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x {sm_max:.0f} MHz",
                "hbm_streaming_equivalent": {
                    "GB_per_s": BYTES_PER_LU_FP32 * lu_batch / (k_ms / 1e3) / 1e9,
                    "frac_of_measured_hbm": BYTES_PER_LU_FP32 * lu_batch / (k_ms / 1e3) / 1e9 / hbm}}

    # --- accuracy of the FP32 form against the FP64 GPU method on the same macro state.
    h64 = HMM(cfg, precision=0)
    Mfix = torch.from_numpy(M0).cuda()
    H32 = h32.micro_batch(Mfix).cpu().numpy()
    H64 = h64.micro_batch(Mfix).cpu().numpy()
    rel = float(np.linalg.norm(H32 - H64, axis=0).max() / np.linalg.norm(H64, axis=0).max())

    # --- plain FP64 method: MPEA steps on the same workload (history set so j >= 2).
    hist = torch.zeros((2, 3, cfg.n_points), dtype=torch.float64, device="cuda")
    h64.set_state(hist, 2)
    M64 = torch.from_numpy(M0).cuda()
    h64.macro_step(M64, 1)
    k64 = max(1, min(args.steps, args.fp64_steps))
    ms64 = timed_steps(lambda: h64.macro_step(M64, 1), k64)
    lu64 = k64 * lu_batch / (ms64 / 1e3)
    h64.close()

    # --- end to end through the C ABI with host buffers (copies inside the timed region).
    Mh = torch.from_numpy(M0).pin_memory().numpy()
    he = HMM(cfg, precision=1)
    he.macro_step_host(Mh, 3)           # start-up steps + graph capture outside the timing
    ke = max(1, min(args.steps, args.e2e_steps))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        he.macro_step_host(Mh, 1)
    e2e_s = time.perf_counter() - t0
    he.close()
    e2e = {"value": world * ke * lu_batch / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": 3 * cfg.n_points * 8, "d2h_bytes_per_step": 3 * cfg.n_points * 8,
           "macro_steps_per_s": ke / e2e_s}

    cpu = None
    if pool is not None:
        oracle_sample(WORKLOAD, 1, args.cpu_workers, pool)   # warm the workers (imports)
        v, info = oracle_sample(WORKLOAD, args.cpu_boxes_per_worker, args.cpu_workers, pool)
        pool.close()
        cpu = {"value": v, "unit": UNIT, "cores": args.cpu_workers, "kind": "oracle",
               "sample": f"{info['boxes']} of the 16384 micro boxes (full 64^2 x 400 steps each), "
                         f"{args.cpu_workers} spawned processes, {info['wall_s']:.1f} s wall"}
    h32.close()

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
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "boxes": cfg.n_points, "micro_nodes": 64,
                       "micro_steps": 400, "lu_per_step": lu_batch, "precision": "fp32-batched",
                       "l2": "flushed (256 MB write) between timed steps",
                       "parallelism": f"replicas x{world}"},
            "macro_steps_per_s": macro_steps_per_s,
            "fp64_plain": {"value": lu64, "unit": UNIT, "macro_steps_per_s": k64 / (ms64 / 1e3),
                           "steps": k64},
            "speedup_fp32_vs_fp64": value / world / lu64,
            "fp32_vs_fp64_rel_err": rel,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": 3 * args.steps,
            "plan_autotuner": plan,
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
           "micro_stepper": ["HeunP", "RK4P"][cfg.micro_stepper], "model": ["field", "flux"][cfg.model],
           "micro_dt_mean": float(h.box_info()["dt"].mean()), "micro_steps": cfg.micro_steps}
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
        h.macro_step(M, 3)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        h.macro_step(M, args.macro_steps)
        t1.record()
        torch.cuda.synchronize()
        sec = t0.elapsed_time(t1) / 1e3
        rec.update(macro_steps=args.macro_steps, macro_steps_per_s=args.macro_steps / sec)
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
    oracle_sample(WORKLOAD, 1, workers, pool)
    for _ in range(args.warmup):
        oracle_sample(WORKLOAD, args.ref_boxes_per_worker, workers, pool)
    tot_lu, tot_s = 0.0, 0.0
    for _ in range(args.steps):
        v, info = oracle_sample(WORKLOAD, args.ref_boxes_per_worker, workers, pool)
        tot_lu += info["lu"]
        tot_s += info["wall_s"]
    pool.close()
    value = tot_lu / tot_s
    sample = (f"each step: {workers * args.ref_boxes_per_worker} of the 16384 micro boxes "
              f"(full 64^2 x 400 steps), {workers} spawned processes")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD_DESC, "precision": "fp64 oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--kernel-reps", type=int, default=3)
    ap.add_argument("--cpu-workers", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--cpu-boxes-per-worker", type=int, default=16)
    ap.add_argument("--ref-boxes-per-worker", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per launch of the dominant kernel, if measured for this build")
    ap.add_argument("--micro-only", action="store_true",
                    help="time hmm_micro_batch alone (see --workload, --macro-grid, --precision, --variant)")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--macro-grid", type=int, nargs="+", default=None)
    ap.add_argument("--box-n", type=int, default=None)
    ap.add_argument("--alpha-micro", type=float, default=None)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--variant", type=int, default=0, help="FP32 kernel: 0 automatic, 1 generic, 2 resident")
    ap.add_argument("--micro-stepper", type=int, default=0, help="with --micro-only: 0 HeunP, 1 RK4P")
    ap.add_argument("--model", type=int, default=0, help="with --micro-only: 0 field model, 1 flux model (FP64)")
    ap.add_argument("--cpu-baseline-micro", action="store_true",
                    help="with --micro-only: also time the oracle on a sample of the boxes")
    ap.add_argument("--no-dns", action="store_true",
                    help="leave the direct-simulation measurement out of the default line")
    ap.add_argument("--dns", action="store_true",
                    help="time the direct simulation (--workload dns_*, --macro-grid for its grid, "
                         "--steps MPEA steps, --fp64-steps for the FP64 form)")
    ap.add_argument("--macro-steps", type=int, default=0,
                    help="with --micro-only: also time this many steady-state macro steps")
    args = ap.parse_args()
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
