"""Pins of the oracle's macro stepper (Section 3.1: RK4P, MPE/MPEA; Section 3.3).

The micro solve is replaced by a cheap surrogate H_avg = a_H D^2_[4] M on the
periodic 1D macro grid (the homogenised operator of Section 2.1 discretised by
the textbook 4th-order central difference), so that the stepper can be
checked against an independent RK4-with-projection integration:
* the midpoint update preserves |M| (to rounding), without projection;
* MPEA converges to the same solution at second order or better (the sign of
  eq. mpe_update, not of the garbled eq. imp_sys, is the consistent one);
* RK4P start-up followed by MPEA is consistent from the first step.
"""
import numpy as np

import workloads as W
from oracle import hmm_oracle as O

AH = np.sqrt(0.75)


def _cfg(n=32):
    return W.config("c1_1d", n_macro=(n, 1, 1), alpha=0.1)


def _surrogate(n):
    DX = 1.0 / n

    def havg(M):
        c = np.array([-1.0, 16.0, -30.0, 16.0, -1.0]) / (12 * DX * DX)
        return AH * sum(ck * np.roll(M, 2 - k, axis=1) for k, ck in enumerate(c))
    return havg


def _rk4p_reference(M0, havg, alpha, T, nsteps):
    M = M0.copy()
    dt = T / nsteps

    def f(M):
        H = havg(M)
        mxH = np.cross(M, H, axis=0)
        return -mxH - alpha * np.cross(M, mxH, axis=0)
    for _ in range(nsteps):
        k1 = f(M)
        k2 = f(M + 0.5 * dt * k1)
        k3 = f(M + 0.5 * dt * k2)
        k4 = f(M + dt * k3)
        M = M + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        M = M / np.linalg.norm(M, axis=0)
    return M


def test_midpoint_update_preserves_norm():
    rng = np.random.default_rng(1)
    M = rng.standard_normal((3, 50))
    M /= np.linalg.norm(M, axis=0)
    h = rng.standard_normal((3, 50)) * 30
    M2 = O.midpoint_update(M, h, 0.05)
    np.testing.assert_allclose(np.linalg.norm(M2, axis=0), 1.0, atol=2e-15)
    # and solves eq. mpe_update: (M2 - M)/dt = -(M + M2)/2 x h
    np.testing.assert_allclose((M2 - M) / 0.05, -np.cross(0.5 * (M + M2), h, axis=0), atol=1e-10)


def test_mpea_converges_to_rk4p():
    n = 32
    cfg = _cfg(n)
    M0 = W.initial_field(cfg)
    havg = _surrogate(n)
    dt0 = O.macro_dt(cfg)
    T = 48 * dt0
    ref = _rk4p_reference(M0, havg, cfg.alpha, T, 48 * 16)
    errs = []
    for s in (1, 2, 4):
        st = O.MacroStepper(cfg, M0, havg=havg, dt=dt0 / s)
        for _ in range(48 * s):
            st.step()
        errs.append(np.abs(st.M - ref).max())
        assert np.abs(np.linalg.norm(st.M, axis=0) - 1.0).max() < 1e-13
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), (errs, rates)
    assert errs[0] < 1e-3


def test_rk4p_startup_steps_match_reference():
    n = 32
    cfg = _cfg(n)
    M0 = W.initial_field(cfg)
    havg = _surrogate(n)
    dt = O.macro_dt(cfg)
    st = O.MacroStepper(cfg, M0, havg=havg, dt=dt)
    st.step()
    st.step()
    ref = _rk4p_reference(M0, havg, cfg.alpha, 2 * dt, 2)
    # the same RK4P except that the stepper normalises its stage states
    assert np.abs(st.M - ref).max() < 1e-6
    assert len(st.hist) == 2 and st.j == 2


def test_default_macro_dt_is_stable_for_mpea():
    n = 32
    cfg = _cfg(n)
    M0 = W.initial_field(cfg)
    st = O.MacroStepper(cfg, M0, havg=_surrogate(n))
    for j in range(200):
        st.step()
    ref = _rk4p_reference(M0, _surrogate(n), cfg.alpha, 200 * st.dt, 200 * 8)
    assert np.abs(st.M - ref).max() < 1e-2
