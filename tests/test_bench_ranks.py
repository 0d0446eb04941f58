"""The N > 1 host logic of bench.py on CPU: two gloo ranks (world size 2) run
independent replicas; the job's time is the slowest rank's and its throughput
counts both ranks' units (weak scaling). No GPU and no data-path collective."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_max, value = bench.aggregate_ranks(times[rank], world, steps=4, units_per_step=1e9, dist=dist)
    out.put((rank, ms_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_total_units():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    times = [120.0, 150.0]
    procs = [mp.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value in res:
        assert ms_max == 150.0
        assert abs(value - 2 * 4 * 1e9 / 0.150) < 1e-6 * value
