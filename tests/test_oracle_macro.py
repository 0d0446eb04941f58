"""Pins of the oracle's macro stepper (Section 3.1: RK4P, MPE/MPEA; Section 3.3).

The micro solve is replaced by a cheap surrogate H_avg = a_H D^2_[4] M on the
periodic 1D macro grid (the homogenised operator of Section 2.1 discretised by
the textbook 4th-order central difference), so that the stepper can be
checked against an independent RK4-with-projection integration:
* the midpoint update preserves |M| (to rounding), without projection;
* MPEA converges to the same solution at second order or better (the sign of
  eq. mpe_update, not of the garbled eq. imp_sys, is the consistent one);
* RK4P start-up followed by MPEA is consistent from the first step;
* the extrapolation coefficients are Adams-Bashforth's: MPEA's h^{j+1/2}
  (eq. h_mpea) is the exact mean of h over the step for h quadratic in t
  (AB3; Section 3.2 links MPEA to AB3), MPE's (eq. h_mpe) for h linear (AB2);
* on the 1D problem MPEA converges at third order in the time step, as the
  paper reports for its 1D example (Section 3.1, Fig. ts), and MPE at second
  order: MPE's coefficients in place of MPEA's fail the third-order pin.
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


def _poly_mean_case(deg, rng):
    """h(t) = sum_k c_k t^k (3-vectors c_k), t_j = 0, t_{j-1} = -dt, t_{j-2} = -2 dt:
    the samples and the exact mean of h over [0, dt]."""
    dt = 0.37
    c = rng.standard_normal((deg + 1, 3, 5))
    h = lambda t: sum(c[k] * t ** k for k in range(deg + 1))
    mean = sum(c[k] * dt ** k / (k + 1) for k in range(deg + 1))
    return h(0.0), [h(-dt), h(-2 * dt)], mean


def test_extrapolation_is_adams_bashforth_mean():
    rng = np.random.default_rng(5)
    for deg in range(3):
        hj, hist, mean = _poly_mean_case(deg, rng)
        np.testing.assert_allclose(O.extrapolate_h(hj, hist, O.MPEA), mean, rtol=0, atol=1e-13)
    for deg in range(2):
        hj, hist, mean = _poly_mean_case(deg, rng)
        np.testing.assert_allclose(O.extrapolate_h(hj, hist, O.MPE), mean, rtol=0, atol=1e-13)
    # one degree higher is not reproduced (the defining order of AB3 and AB2)
    hj, hist, mean = _poly_mean_case(3, rng)
    assert np.abs(O.extrapolate_h(hj, hist, O.MPEA) - mean).max() > 1e-3
    hj, hist, mean = _poly_mean_case(2, rng)
    assert np.abs(O.extrapolate_h(hj, hist, O.MPE) - mean).max() > 1e-3


def _order_study(scheme, n=32, alpha=0.01, steps=(48, 96, 192)):
    """RMS error at T = 48 default macro steps against the RK4P reference, at
    the step counts given; returns (errors, observed rates)."""
    cfg = W.config("c1_1d", n_macro=(n, 1, 1), alpha=alpha)
    M0 = W.initial_field(cfg)
    havg = _surrogate(n)
    T = 48 * O.macro_dt(cfg)
    ref = _rk4p_reference(M0, havg, alpha, T, 48 * 64)
    errs = []
    for s in steps:
        st = O.MacroStepper(cfg, M0, havg=havg, dt=T / s, scheme=scheme)
        for _ in range(s):
            st.step()
        errs.append(np.sqrt(np.mean((st.M - ref) ** 2)))
    errs = np.array(errs)
    return errs, np.log2(errs[:-1] / errs[1:])


def test_mpea_third_order_in_1d():
    errs, rates = _order_study(O.MPEA)
    assert np.all(rates >= 2.7), (errs, rates)


def test_mpe_second_order_in_1d():
    errs, rates = _order_study(O.MPE)
    assert np.all((rates > 1.8) & (rates < 2.3)), (errs, rates)
    # and it is less accurate than MPEA at every step size (Section 3.1, Fig. ts)
    assert np.all(errs > _order_study(O.MPEA)[0])


def test_mpe_startup_is_one_rk4p_step():
    n = 32
    cfg = _cfg(n).replace(macro_stepper=1)
    M0 = W.initial_field(cfg)
    havg = _surrogate(n)
    st = O.MacroStepper(cfg, M0, havg=havg)
    assert st.scheme == O.MPE and st.n_startup == 1
    st.step()
    ref = _rk4p_reference(M0, havg, cfg.alpha, st.dt, 1)
    assert np.abs(st.M - ref).max() < 1e-6
    M1, h0 = st.M.copy(), st.hist[0].copy()
    st.step()
    # the second step is an MPE step: h^1 from M^1, then the midpoint update with
    # 3/2 h^1 - 1/2 h^0 (eqs. h_mpe, mpe_update)
    h1 = O.h_term(M1, havg(M1), cfg.alpha)
    np.testing.assert_allclose(st.hist[0], h1, rtol=0, atol=1e-12 * np.abs(h1).max())
    np.testing.assert_allclose(st.M, O.midpoint_update(M1, 1.5 * h1 - 0.5 * h0, st.dt), rtol=0, atol=1e-14)
