"""GPU parity of the direct simulation (include/hmm_dns.h) against the oracle.

Whole-grid cases compare every point after a number of steps that covers the
RK4P start-up, the first MPEA steps (history rotation, state ping-pong) and a
longer run; grids span several warp strips (26 nodes per strip at order 4, 30
at order 2) with ragged last strips, fewer columns than one warp, and several
row chunks. The benchmark's full grid (1500^2, eq. coeff_quasi) is compared
at sampled points whose patch the oracle computes one by one.

Bounds: max over points of |M_gpu - M_ref|_2 (|M| = 1) below 1e-12 for the
FP64 form and 1e-6 for the float-float FP32 form.
"""
import numpy as np
import pytest

import workloads as W
from oracle import dns_oracle as D

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


def _cfg(n, order=4, alpha=0.05, name=None):
    base = W.dns_config(name or ("dns_quasi2d" if len(n) == 2 else "dns_loc1d"))
    return base.replace(n=tuple(n) + (1,) * (3 - len(n)), alpha=alpha, stencil_order=order)


def _err(Mg, Mr):
    return float(np.linalg.norm(np.asarray(Mg) - Mr, axis=0).max())


def _gpu(torch, cfg, M0, steps, precision, face_table=None, calls=None):
    from paper_2108_09463_gb300 import DNS
    d = DNS(cfg, precision=precision, face_table=face_table)
    M = torch.from_numpy(np.ascontiguousarray(M0)).cuda()
    for n in (calls or [steps]):
        d.step(M, n)
    info = d.info()
    d.close()
    return M.cpu().numpy(), info


CASES = [
    ((100,), 4, 12), ((67,), 2, 12), ((20,), 4, 5),
    ((40, 37), 4, 12), ((13, 9), 4, 6), ((33, 50), 2, 12), ((64, 64), 4, 3), ((70, 29), 4, 1),
    ((8, 100), 4, 4), ((100, 8), 2, 4),
]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "ff32"])
@pytest.mark.parametrize("n,order,steps", CASES, ids=[f"{'x'.join(map(str, c[0]))}-o{c[1]}-s{c[2]}" for c in CASES])
def test_dns_parity(torch_cuda, n, order, steps, precision):
    cfg = _cfg(n, order)
    M0 = W.dns_initial(cfg, noise=0.2, seed=len(n) * 100 + n[0])
    Mg, info = _gpu(torch_cuda, cfg, M0, steps, precision)
    assert abs(info["dt"] - D.dns_dt(cfg)) <= 1e-9 * info["dt"]
    assert info["j"] == steps
    ref = D.DNS(cfg, M0, dt=info["dt"])
    ref.step(steps)
    e = _err(Mg, ref.M)
    assert e < TOL[precision], (n, order, steps, precision, e)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "ff32"])
def test_dns_long_run(torch_cuda, precision):
    cfg = _cfg((64, 48), 4, alpha=0.01)
    M0 = W.dns_initial(cfg, noise=0.1, seed=5)
    Mg, info = _gpu(torch_cuda, cfg, M0, 200, precision)
    ref = D.DNS(cfg, M0, dt=info["dt"])
    ref.step(200)
    e = _err(Mg, ref.M)
    assert e < TOL[precision], (precision, e)
    assert np.abs(np.linalg.norm(Mg, axis=0) - 1).max() < (1e-13 if precision == 0 else 1e-6)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "ff32"])
def test_dns_calls_continue_one_trajectory(torch_cuda, precision):
    cfg = _cfg((30, 41), 4)
    M0 = W.dns_initial(cfg, noise=0.2, seed=11)
    # one call of 33 steps (graph replays of six) against calls that start the
    # six-step graphs at other phases of the state ping-pong and history ring
    M1, _ = _gpu(torch_cuda, cfg, M0, 33, precision)
    M2, info = _gpu(torch_cuda, cfg, M0, 33, precision, calls=[1, 0, 3, 5, 7, 11, 6])
    assert info["j"] == 33
    assert np.abs(M1 - M2).max() <= (0.0 if precision == 0 else 1e-15)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "ff32"])
def test_dns_face_table(torch_cuda, precision):
    """Tabulated coefficient (eq. coeff_loc2D) against the oracle on the same faces."""
    cfg = W.dns_config("dns_loc2d", n=(48, 40, 1))
    af = D.face_coefficients(cfg)
    table = np.concatenate([a.ravel() for a in af])
    M0 = W.dns_initial(cfg, noise=0.1, seed=3)
    Mg, info = _gpu(torch_cuda, cfg, M0, 10, precision, face_table=table)
    assert abs(info["dt"] - D.dns_dt(cfg)) <= 1e-9 * info["dt"]
    ref = D.DNS(cfg, M0, dt=info["dt"])
    ref.step(10)
    e = _err(Mg, ref.M)
    assert e < TOL[precision], (precision, e)


def test_dns_host_variant_and_zero_steps(torch_cuda):
    from paper_2108_09463_gb300 import DNS
    cfg = _cfg((24, 30), 4)
    M0 = W.dns_initial(cfg, noise=0.2, seed=1)
    Md, _ = _gpu(torch_cuda, cfg, M0, 5, 1)
    d = DNS(cfg, precision=1)
    Mh = M0.copy()
    d.step_host(Mh, 0)
    assert np.array_equal(Mh, M0)
    d.step_host(Mh, 5)
    d.close()
    assert np.abs(Mh - Md).max() == 0.0


def test_dns_nonfinite_reported(torch_cuda):
    from paper_2108_09463_gb300 import DNS, HmmError
    cfg = _cfg((16, 40), 4)
    M0 = W.dns_initial(cfg)
    M0[0, 77] = np.nan
    d = DNS(cfg, precision=1)
    M = torch_cuda.from_numpy(M0).cuda()
    with pytest.raises(HmmError) as ei:
        d.step(M, 4)
    assert ei.value.status == 6
    d.close()


@pytest.mark.parametrize("precision", [1, 0], ids=["ff32", "fp64"])
def test_dns_full_size_sampled(torch_cuda, precision):
    """The benchmark's grid (eq. coeff_quasi, dx = 1/1500, (EX2) data), in the
    launch configuration the benchmark times, at sampled points after the
    start-up and four MPEA steps."""
    cfg = W.dns_config("dns_quasi2d")
    M0 = W.dns_initial(cfg)
    steps = 6
    Mg, info = _gpu(torch_cuda, cfg, M0, steps, precision)
    n = cfg.shape
    rng = np.random.default_rng(2)
    pts = [(0, 0), (n[0] - 1, n[1] - 1), (0, n[1] - 1), (749, 1499), (1000, 26 * 37)]
    pts += [tuple(int(v) for v in rng.integers(0, n[0], 2)) for _ in range(3)]
    Mg = Mg.reshape((3,) + n)
    for c in pts:
        ref = D.patch_run(cfg, M0, c, steps, info["dt"])
        e = float(np.linalg.norm(Mg[:, c[0], c[1]] - ref))
        assert e < TOL[precision], (c, precision, e)


def test_dns_plan_autotuned(torch_cuda):
    """The first MPEA step autotunes the chunk length among the one-wave plan,
    half, twice and four times it; the results do not depend on the plan."""
    from paper_2108_09463_gb300 import DNS
    cfg = _cfg((300, 260), 4)
    M0 = W.dns_initial(cfg, noise=0.1, seed=4)
    d = DNS(cfg, precision=1)
    p0 = d.plan()
    M = torch_cuda.from_numpy(M0.copy()).cuda()
    d.step(M, 2)                       # start-up only: no tuning yet
    assert d.plan() == p0
    d.step(M, 7)
    p1 = d.plan()
    d.close()
    c1 = p0["chunk"]
    assert p1["chunk"] in {c1, max(8, c1 // 2), min(300, 2 * c1), min(300, 4 * c1)}
    assert p1["items"] == p1["strips"] * ((300 + p1["chunk"] - 1) // p1["chunk"])
    M2, _ = _gpu(torch_cuda, cfg, M0, 9, 1)
    assert np.abs(M.cpu().numpy() - M2).max() == 0.0
