"""GPU test of hmm_micro_batch_noalloc, the allocation-free micro batch.

That entry point exists for callers that must not allocate device memory (an
allocator's own callbacks, where cudaMalloc would re-enter the allocator, and
applications whose device memory another framework has reserved). It must give
the same H_avg as the regular entry point, call after call, although every call
reuses one fixed scratch array inside the library: in 2D, in 3D with boxes so
large that only a few per-CTA arenas fit the array (a reduced grid whose CTAs
index the arenas by block), in 1D with the RK4P micro stepper and in 2D with MPEA.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-6      # the batched FP32 form's bound, as in tests/test_gpu_parity.py


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_09463_gb300 import build
    build()
    return torch


def _rel(a, b):
    return np.linalg.norm(a - b, axis=0).max() / np.linalg.norm(b, axis=0).max()


def test_noalloc_matches_regular_entry_point_twice(torch_cuda):
    from paper_2108_09463_gb300 import HMM, micro_batch_noalloc
    torch = torch_cuda
    cfg = W.config("c2_2d", n_macro=(12, 12, 1), box_n=32, micro_steps=60)
    fields = [W.fourier_field(cfg, seed).reshape(3, -1) for seed in (11, 12)]
    h = HMM(cfg, precision=1)
    for i, M0 in enumerate(fields):
        M = torch.from_numpy(np.ascontiguousarray(M0)).cuda()
        ref = h.micro_batch(M).cpu().numpy()
        out = torch.full_like(M, float("nan"))
        free_before = torch.cuda.mem_get_info()[0]
        micro_batch_noalloc(cfg, M, out)
        torch.cuda.synchronize()
        if i == 1:   # the scratch array exists since the first call: nothing new is allocated
            assert torch.cuda.mem_get_info()[0] == free_before
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert _rel(got, ref) < TOL_FP32, (i, _rel(got, ref))
    h.close()


def test_noalloc_rejects_sizes_beyond_its_maximum(torch_cuda):
    from paper_2108_09463_gb300 import HmmError, micro_batch_noalloc
    torch = torch_cuda
    cfg = W.config("c2_2d", n_macro=(8, 8, 1), box_n=24, micro_steps=20000)
    M = torch.from_numpy(W.initial_field(cfg)).cuda()
    out = torch.empty_like(M)
    with pytest.raises(HmmError) as ei:
        micro_batch_noalloc(cfg, M, out)
    assert ei.value.status == 1 and "micro_steps" in str(ei.value)
    big = W.config("c4_3d", n_macro=(5, 5, 5), box_n=64, mu_over_eps=4.0, micro_steps=10)
    M = torch.from_numpy(W.initial_field(big)).cuda()
    with pytest.raises(HmmError) as ei:
        micro_batch_noalloc(big, M, torch.empty_like(M))
    assert ei.value.status == 1 and "maximum" in str(ei.value)


def _compare_twice(torch, cfg, seeds, kernel_variant=0):
    from paper_2108_09463_gb300 import HMM, micro_batch_noalloc
    h = HMM(cfg, precision=1, kernel_variant=kernel_variant)
    for seed in seeds:
        M0 = W.fourier_field(cfg, seed).reshape(3, -1)
        M = torch.from_numpy(np.ascontiguousarray(M0)).cuda()
        ref = h.micro_batch(M).cpu().numpy()
        out = torch.full_like(M, float("nan"))
        micro_batch_noalloc(cfg, M, out)
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert _rel(got, ref) < TOL_FP32, (cfg.dim, seed, _rel(got, ref))
    h.close()


def test_noalloc_3d_reduced_grid(torch_cuda):
    # 40^3 boxes: each per-CTA arena is about 10.75 MB, so only two fit the 32 MiB
    # array and the launch runs two CTAs over 125 boxes
    cfg = W.config("c4_3d", n_macro=(5, 5, 5), box_n=40, micro_steps=20)
    _compare_twice(torch_cuda, cfg, (21, 22), kernel_variant=1)


def test_noalloc_1d_rk4p(torch_cuda):
    cfg = W.config("c1_1d", n_macro=(16, 1, 1), micro_steps=100, micro_stepper=1)
    _compare_twice(torch_cuda, cfg, (31, 32))


def test_noalloc_2d_mpea(torch_cuda):
    # the multi-step stepper's per-node history arrays enlarge each arena
    cfg = W.config("c2_2d", n_macro=(6, 6, 1), box_n=32, micro_steps=40, alpha_micro=0.1, micro_stepper=3)
    _compare_twice(torch_cuda, cfg, (33, 34), kernel_variant=1)


def test_noalloc_refuses_a_capturing_stream(torch_cuda):
    from paper_2108_09463_gb300 import HmmError, micro_batch_noalloc
    torch = torch_cuda
    cfg = W.config("c2_2d", n_macro=(8, 8, 1), box_n=24, micro_steps=20)
    M = torch.from_numpy(W.initial_field(cfg)).cuda()
    out = torch.empty_like(M)
    x = torch.zeros(16, device="cuda")
    g = torch.cuda.CUDAGraph()
    refused = None
    with torch.cuda.graph(g):
        x.add_(1.0)
        try:
            micro_batch_noalloc(cfg, M, out)
        except HmmError as e:
            refused = e
    # the capture ended normally and the graph replays
    g.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
    assert refused is not None and refused.status == 1 and "captured" in str(refused)
    # and the entry point works again outside the capture
    micro_batch_noalloc(cfg, M, out)
    assert np.all(np.isfinite(out.cpu().numpy()))
