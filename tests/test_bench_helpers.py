"""Host-side helpers of bench.py (no GPU): the roofline's DRAM-traffic figure is
taken from a committed ncu record only while the kernel source it was captured
from is unchanged, and the benchmark's workload table is consistent with the
workload definitions."""
import os
import shutil

import bench
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_record_applies_only_to_its_source(tmp_path):
    for name, spec in bench.WORKLOADS.items():
        if not spec["traffic"]:
            continue
        rec = os.path.join(ROOT, "profiles", spec["traffic"])
        src = os.path.join(ROOT, "paper_2108_09463_gb300", "csrc", spec["source"])
        value = bench._traffic_from_profile(rec, src)
        assert value is None or value > 0
        # one byte more in the source: the record no longer applies
        changed = tmp_path / os.path.basename(src)
        shutil.copy(src, changed)
        with open(changed, "a") as f:
            f.write("\n")
        assert bench._traffic_from_profile(rec, str(changed)) is None
    assert bench._traffic_from_profile(None, "x") is None


def test_benchmark_workloads_match_their_definitions():
    for name, spec in bench.WORKLOADS.items():
        cfg = W.config(name)
        assert f"{cfg.micro_steps} HeunP micro steps" in spec["desc"], name
        waves = spec.get("waves", 1)
        assert cfg.n_points % waves == 0
        # a wave step of the headline workload holds a whole number of boxes per wave
        if waves > 1:
            assert cfg.box_n_field is None and cfg.eps_field is None
    assert bench.WORKLOAD in bench.WORKLOADS
    assert set(bench.SUB_WORKLOADS) <= set(bench.WORKLOADS)
