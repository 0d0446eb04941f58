"""Pins of the oracle's multi-step micro steppers MPE and MPEA (Section 3.1) and of
their time-step rule (Section 3.2).

* The stability rule takes the related Adams-Bashforth methods (AB2 for MPE, AB3 for
  MPEA, eq. mpe_update_ab): their textbook real-axis limits (1 and 6/11), AB3's
  imaginary-axis limit from the boundary locus z = rho(e^{i theta}) / sigma(e^{i theta})
  (an independent construction, about 0.7236), and AB2's vanishing imaginary interval
  (|zeta|^2 = 1 - 2 alpha s + s^4/2 + ..., so s_max -> (4 alpha)^(1/3)).
* The midpoint update (eq. mpe_update) solved per node satisfies its defining equation
  and keeps |m| (the Cayley transform is a rotation).
* The start-up steps are RK4P's; afterwards MPE converges at second order and MPEA at
  third order on this 1D problem, as the paper observes in 1D (Section 3.1, Fig. ts),
  with smaller errors; |m| = 1 throughout.
* At low damping MPEA's stability limit beats HeunP's and per stencil evaluation it is
  the cheapest of the four (Section 3.2, Fig. stab_cost).
"""
import numpy as np
import pytest

import workloads as W
from oracle import hmm_oracle as O


def test_adams_bashforth_real_axis_limits():
    a = 1e4
    assert abs(O.stability_limit(a, O.MICRO_MPE) * abs(complex(-a, 1.0)) - 1.0) < 1e-4
    assert abs(O.stability_limit(a, O.MICRO_MPEA) * abs(complex(-a, 1.0)) - 6.0 / 11.0) < 1e-4


def test_ab3_imaginary_limit_from_boundary_locus():
    th = np.linspace(1e-4, np.pi, 200001)
    zeta = np.exp(1j * th)
    z = (zeta ** 3 - zeta ** 2) / ((23 * zeta ** 2 - 16 * zeta + 5) / 12)
    # the first crossing of the imaginary axis away from z = 0
    k = np.nonzero(np.diff(np.sign(z.real)))[0][0]
    t = z.real[k] / (z.real[k] - z.real[k + 1])
    y = z.imag[k] + t * (z.imag[k + 1] - z.imag[k])
    assert abs(y - 0.7236) < 1e-3
    assert abs(O.stability_limit(1e-9, O.MICRO_MPEA) - y) < 1e-5


def test_ab2_has_no_imaginary_interval():
    for a in (1e-6, 8e-6):
        assert abs(O.stability_limit(a, O.MICRO_MPE) - (4 * a) ** (1 / 3)) < 0.02 * (4 * a) ** (1 / 3)


def test_midpoint_solve_satisfies_the_update():
    rng = np.random.default_rng(7)
    m = rng.normal(size=(2, 3, 5, 4))
    h = 50 * rng.normal(size=(2, 3, 5, 4))
    dt = 0.02
    mp = O.midpoint_solve(m, h, dt, 1)
    res = (mp - m) / dt + np.cross(0.5 * (m + mp), h, axis=1)
    assert np.abs(res).max() < 1e-12 * np.abs(h).max()
    assert np.abs(np.linalg.norm(mp, axis=1) - np.linalg.norm(m, axis=1)).max() < 1e-14


def _box(alpha_micro=0.1):
    cfg = W.config("c1_1d", n_macro=(16, 1, 1), box_n=41, micro_steps=10, alpha_micro=alpha_micro)
    M0 = W.initial_field(cfg)
    geo = O.box_geometry(cfg, 5)
    mi = O.micro_initial(cfg, M0, geo)[None]
    af = [a[None] for a in O.face_coefficients(cfg, geo)]
    N, r = geo["N"], geo["r"]
    Wd = O.space_weights(N, geo["dx"], geo["mu"], cfg.px, cfg.qx)[r:N - r]
    return cfg, geo, mi, af, Wd


def _final(cfg, geo, mi, af, Wd, T, nsteps, stepper):
    w = np.zeros(nsteps + 1)
    _, m, _, nd = O.micro_solve(mi, af, geo["dx"], T / nsteps, nsteps, cfg.alpha_micro, Wd, w, 4,
                                trace=True, stepper=stepper)
    return m, nd


@pytest.mark.parametrize("stepper,n_start", [(O.MICRO_MPE, 1), (O.MICRO_MPEA, 2)])
def test_startup_steps_are_rk4p(stepper, n_start):
    cfg, geo, mi, af, Wd = _box()
    dt = 0.5 * geo["dt"]
    a, _ = _final(cfg, geo, mi, af, Wd, n_start * dt, n_start, stepper)
    b, _ = _final(cfg, geo, mi, af, Wd, n_start * dt, n_start, O.RK4P)
    assert np.array_equal(a, b)
    a, _ = _final(cfg, geo, mi, af, Wd, (n_start + 1) * dt, n_start + 1, stepper)
    b, _ = _final(cfg, geo, mi, af, Wd, (n_start + 1) * dt, n_start + 1, O.RK4P)
    assert 0 < np.abs(a - b).max() < 1e-2 * np.abs(b - mi).max()


def test_mpe_second_order_mpea_third_order_in_1d():
    cfg, geo, mi, af, Wd = _box()
    T = 40 * geo["dt"]
    ref, _ = _final(cfg, geo, mi, af, Wd, T, 40 * 64, O.RK4P)
    errs = {}
    for st in (O.MICRO_MPE, O.MICRO_MPEA):
        e = []
        for s in (2, 4, 8):
            m, nd = _final(cfg, geo, mi, af, Wd, T, 40 * s, st)
            assert nd.max() < 1e-13   # Cramer rounding only: no projection
            e.append(np.abs(m - ref).max())
        errs[st] = np.array(e)
    r_mpe = np.log2(errs[O.MICRO_MPE][:-1] / errs[O.MICRO_MPE][1:])
    r_mpea = np.log2(errs[O.MICRO_MPEA][:-1] / errs[O.MICRO_MPEA][1:])
    assert np.all(r_mpe > 1.8) and np.all(r_mpe < 2.3), (errs, r_mpe)
    assert np.all(r_mpea > 2.7), (errs, r_mpea)
    assert np.all(errs[O.MICRO_MPEA] < errs[O.MICRO_MPE]), errs


def test_low_damping_cost_per_unit_time():
    """Stencil evaluations per unit of micro time ~ stages / s_max: at alpha = 0.01
    MPEA and RK4P cost about the same and HeunP and MPE more (Section 3.2)."""
    cost = {st: stages / O.stability_limit(0.01, st)
            for st, stages in ((O.HEUNP, 2), (O.RK4P, 4), (O.MICRO_MPE, 1), (O.MICRO_MPEA, 1))}
    assert abs(cost[O.MICRO_MPEA] / cost[O.RK4P] - 1.0) < 0.1
    assert cost[O.HEUNP] > 2 * cost[O.MICRO_MPEA] and cost[O.MICRO_MPE] > 2 * cost[O.MICRO_MPEA]
    # high damping: HeunP is the cheapest
    hi = {st: stages / O.stability_limit(1.2, st)
          for st, stages in ((O.HEUNP, 2), (O.RK4P, 4), (O.MICRO_MPE, 1), (O.MICRO_MPEA, 1))}
    assert min(hi, key=hi.get) == O.HEUNP


def test_micro_batch_mpea_close_to_rk4p():
    """At the same micro time and a small step, MPEA and RK4P give the same average."""
    cfg = W.config("c1_1d", n_macro=(16, 1, 1), box_n=81, micro_steps=120, dt_safety=0.3, micro_stepper=1,
                   alpha_micro=0.1)
    M0 = W.initial_field(cfg)
    H1 = O.micro_batch(cfg, M0, points=[3, 9])
    dt1 = O.micro_dt(cfg, cfg.eps / cfg.pts_per_eps)
    cfg3 = cfg.replace(micro_stepper=3)
    dt3 = O.micro_dt(cfg3, cfg.eps / cfg.pts_per_eps)
    steps = int(round(120 * dt1 / dt3)) * 2
    cfg3 = cfg3.replace(micro_steps=steps, dt_safety=cfg.dt_safety * dt1 * 120 / (steps * dt3))
    H3 = O.micro_batch(cfg3, M0, points=[3, 9])
    assert np.abs(H3 - H1).max() < 1e-3 * np.abs(H1).max(), (H1, H3)
