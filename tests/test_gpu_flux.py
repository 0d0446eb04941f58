"""GPU parity of the flux model (Section 2.2, eq. macro_flux) against the oracle.

The FP64 form is compared with the flux oracle evaluated in long double on
sampled boxes (the raw flux columns, bound 1e-12 relative to the largest
column), the batched FP32 form with the FP64 oracle on every box (bound 1e-6);
the macro divergence that hmm_micro_batch returns for a flux-model handle
against the oracle's divergence of the same columns, and the macro steps
against the oracle's flux-model stepper over the RK4P start-up and MPEA steps.
"""
import numpy as np
import pytest

import workloads as W
from oracle import flux_oracle as F

pytestmark = pytest.mark.gpu

TOL = 1e-12
ORACLE_FP64_FLOOR = 3e-12


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_09463_gb300 import build
    build()
    return torch


CASES = {
    "1d": ("c1_1d", dict(n_macro=(12, 1, 1), box_n=81, micro_steps=60)),
    "1d_order2_interp2": ("c1_1d", dict(n_macro=(12, 1, 1), box_n=61, micro_steps=50, stencil_order=2,
                                        interp_order=2)),
    "2d": ("c2_2d", dict(n_macro=(8, 8, 1), box_n=24, micro_steps=40)),
    "2d_ragged": ("c2_2d", dict(n_macro=(6, 7, 1), box_n=37, micro_steps=23)),
    "2d_order2_rk4p": ("c2_2d", dict(n_macro=(8, 8, 1), box_n=24, micro_steps=30, stencil_order=2,
                                     micro_stepper=1)),
    "2d_slow_fast": ("c3_2d_uneven", dict(n_macro=(8, 8, 1), eps_field=None, box_n_field=None,
                                          eps=1 / 250, box_n=32, micro_steps=30, precision=0)),
    "3d": ("c4_3d", dict(n_macro=(5, 5, 6), box_n=16, mu_over_eps=0.9, micro_steps=20, precision=0)),
    "3d_n32": ("c4_3d", dict(n_macro=(5, 5, 5), box_n=32, micro_steps=12, precision=0)),
    "2d_order2": ("c2_2d", dict(n_macro=(8, 8, 1), box_n=24, micro_steps=30, stencil_order=2)),
    # uneven boxes (N = 32..96 by the uneven workload's field 1/eps = 250 + 150 sin 2 pi x1 cos 2 pi x2,
    # on an 8 x 8 grid): packs and clusters
    "2d_uneven": ("c3_2d_uneven", dict(n_macro=(8, 8, 1), micro_steps=12, precision=0)),
    # edge sizes: the smallest order-4 box (N = 2r + 2, three weighted faces per axis) and
    # the fewest micro steps with a non-zero time average (M = 2)
    "2d_min_box": ("c2_2d", dict(n_macro=(6, 5, 1), box_n=8, mu_over_eps=0.15, micro_steps=20)),
    "2d_two_micro_steps": ("c2_2d", dict(n_macro=(6, 6, 1), box_n=24, micro_steps=2)),
}


def _cfg(case):
    name, over = CASES[case]
    cfg = W.config(name, **over).replace(model=1)
    if name == "c3_2d_uneven" and "eps_field" in over:
        cfg = cfg.replace(eps_field=None, box_n_field=None)
    return cfg


def _points(cfg, k=4):
    P = cfg.n_points
    return sorted(set([0, P - 1, P // 2, P // 3]))[:k]


# FP32: the 2D and 3D HeunP cases run on the resident kernels (chosen automatically),
# the others on the generic kernel; "_generic" forces the generic kernel.
FP32_CASES = sorted(CASES) + ["2d_generic", "2d_ragged_generic", "3d_generic"]


@pytest.mark.parametrize("case", FP32_CASES)
def test_flux_columns_parity_fp32(torch_cuda, case):
    from paper_2108_09463_gb300 import HMM
    variant = 1 if case.endswith("_generic") else 0
    cfg = _cfg(case.replace("_generic", ""))
    M0 = W.initial_field(cfg)
    h = HMM(cfg, precision=1, kernel_variant=variant)
    M = torch_cuda.from_numpy(M0).cuda()
    Fg = h.flux_batch(M).cpu().numpy()
    H = h.micro_batch(M).cpu().numpy()
    h.close()
    Fr = F.micro_batch_flux(cfg, M0)
    err = np.abs(Fg - Fr).max() / np.abs(Fr).max()
    assert err < 1e-6, (case, err)
    Hr = F.flux_divergence(cfg, Fg)
    assert np.abs(H - Hr).max() <= 1e-13 * np.abs(Hr).max()


@pytest.mark.parametrize("case", sorted(CASES))
def test_flux_columns_parity(torch_cuda, case):
    from paper_2108_09463_gb300 import HMM
    cfg = _cfg(case)
    M0 = W.initial_field(cfg)
    h = HMM(cfg, precision=0)
    M = torch_cuda.from_numpy(M0).cuda()
    Fg = h.flux_batch(M).cpu().numpy()
    H = h.micro_batch(M).cpu().numpy()
    h.close()
    assert np.all(np.isfinite(Fg))
    pts = _points(cfg, 2 if cfg.dim == 3 else 4)
    Fr = F.micro_batch_flux(cfg, M0, points=pts, dtype=np.longdouble)
    scale = np.abs(Fr.astype(np.float64)).max()
    err = np.abs(Fg[:, :, pts] - Fr.astype(np.float64)).max() / scale
    assert err < TOL, (case, err)
    # the divergence hmm_micro_batch returns for a flux-model handle
    Hr = F.flux_divergence(cfg, Fg)
    assert np.abs(H - Hr).max() <= 1e-13 * np.abs(Hr).max()


def test_flux_field_against_oracle(torch_cuda):
    """div F_avg on every macro point against the oracle's flux field (FP64)."""
    from paper_2108_09463_gb300 import HMM
    cfg = _cfg("2d")
    M0 = W.initial_field(cfg)
    h = HMM(cfg, precision=0)
    H = h.micro_batch(torch_cuda.from_numpy(M0).cuda()).cpu().numpy()
    h.close()
    Hr = F.flux_field(cfg, M0)
    err = np.linalg.norm(H - Hr, axis=0).max() / np.linalg.norm(Hr, axis=0).max()
    assert err < TOL + ORACLE_FP64_FLOOR, err


def test_flux_macro_steps(torch_cuda):
    from paper_2108_09463_gb300 import HMM
    cfg = _cfg("1d")
    M0 = W.initial_field(cfg)
    h = HMM(cfg, precision=0)
    M = torch_cuda.from_numpy(M0).cuda()
    nsteps = 4
    h.macro_step(M, nsteps)
    Mg = M.cpu().numpy()
    st = F.macro_stepper(cfg, M0, dt=h.macro_dt())
    hmax = np.linalg.norm(st.havg(M0), axis=0).max()
    for _ in range(nsteps):
        st.step()
    err = np.abs(Mg - st.M).max()
    bound = 4 * nsteps * h.macro_dt() * (TOL + ORACLE_FP64_FLOOR) * hmax + 1e-14
    assert err < bound, (err, bound)
    assert np.abs(np.linalg.norm(Mg, axis=0) - 1).max() < 1e-13
    h.close()


def test_flux_model_validation(torch_cuda):
    from paper_2108_09463_gb300 import HMM, HmmError
    with pytest.raises(HmmError):
        HMM(_cfg("1d"), precision=1, kernel_variant=2)   # no 1D resident kernel
    cfg = _cfg("2d")
    HMM(cfg, precision=1, kernel_variant=2).close()      # the resident kernels take the flux
    h = HMM(cfg.replace(model=0), precision=0)
    with pytest.raises(HmmError):
        h.flux_batch(torch_cuda.from_numpy(W.initial_field(cfg)).cuda())
    h.close()
