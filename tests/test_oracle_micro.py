"""Pins of the oracle's micro solve and averaging (Sections 2.2-2.3, 3.1, 4.1-4.2).

* HeunP keeps |m| = 1 on the interior and m = m_init on the Dirichlet ring.
* The exchange energy decays monotonically for alpha > 0 under the dt rule,
  and the solve blows up above the HeunP stability limit (eq. Cstab).
* HeunP is second order in dt (Section 3.1).
* Physics: H_avg approaches div(grad m_init(0) A^H) (Theorem 2) with A^H from
  closed forms: the 1D harmonic mean (EX1 coefficient) with the paper's 1D
  parameters (Section 5, locally periodic example: mu = 3.9 eps, mu' = 8 eps,
  eta ~ eps^2, alpha = 1.2) and the separable (EX3) coefficient in 2D.
* Invariants: constant M gives H_avg = 0; rotating all macro vectors rotates H_avg.
* The error's dependence on eps (Section 4.4, length of the time interval eta): with
  mu, mu' and eta large enough that the other contributions are small, the
  remaining error E_eps of the (EX2) micro problem falls by about four when eps is
  halved (E_eps <= C eps^2), with A^H from the cell problem; on the averaging
  width mu (Section 4.4, averaging domain size): steep while mu is a few eps, flat
  from about 3.5 eps; on the averaging time eta: steep while eta is a few eps^2; and on
  the box half-width mu': falling until the boundary error is below the rest.
"""
import functools

import numpy as np
import pytest

import workloads as W
from oracle import cell_problem as C
from oracle import hmm_oracle as O


def _one_box(cfg, p, M0):
    geo = O.box_geometry(cfg, p)
    mi = O.micro_initial(cfg, M0, geo)[None]
    af = [a[None] for a in O.face_coefficients(cfg, geo)]
    N, r = geo["N"], geo["r"]
    W1 = O.space_weights(N, geo["dx"], geo["mu"], cfg.px, cfg.qx)[r:N - r]
    Wd = W1
    for _ in range(cfg.dim - 1):
        Wd = np.multiply.outer(Wd, W1)
    w = O.time_weights(cfg.micro_steps, cfg.pt, cfg.qt)
    return geo, mi, af, Wd, w


@pytest.mark.parametrize("name,over", [("c1_1d", dict(n_macro=(16, 1, 1), box_n=81, micro_steps=120)),
                                       ("c2_2d", dict(n_macro=(8, 8, 1), box_n=24, micro_steps=60))])
def test_norm_ring_and_energy(name, over):
    cfg = W.config(name, **over)
    M0 = W.initial_field(cfg)
    geo, mi, af, Wd, w = _one_box(cfg, 3, M0)
    S, m, E, nd = O.micro_solve(mi, af, geo["dx"], geo["dt"], cfg.micro_steps, cfg.alpha_micro,
                                Wd, w, cfg.stencil_order, trace=True)
    assert nd.max() < 1e-14
    r = geo["r"]
    ring = np.ones(m.shape, bool)
    ring[(Ellipsis,) + tuple(slice(r, geo["N"] - r) for _ in range(cfg.dim))] = False
    assert np.array_equal(m[ring], mi[ring])
    E = E[:, 0]
    assert np.all(np.diff(E) <= 1e-13 * E[0]), "energy must decay monotonically for alpha > 0"
    assert E[-1] < E[0]


def test_unstable_above_heun_limit():
    for safety, stable in ((0.8, True), (1.3, False)):
        cfg = W.config("c1_1d", n_macro=(16, 1, 1), box_n=81, micro_steps=300, dt_safety=safety)
        M0 = W.initial_field(cfg)
        geo, mi, af, Wd, w = _one_box(cfg, 3, M0)
        _, _, E, _ = O.micro_solve(mi, af, geo["dx"], geo["dt"], cfg.micro_steps, cfg.alpha_micro,
                                   Wd, w, 4, trace=True)
        grow = E.max() / E[0]
        assert (grow <= 1.0 + 1e-12) if stable else (grow > 10.0), (safety, grow)


def test_heun_second_order_in_time():
    cfg = W.config("c1_1d", n_macro=(16, 1, 1), box_n=41, micro_steps=10)
    M0 = W.initial_field(cfg)
    geo, mi, af, Wd, _ = _one_box(cfg, 5, M0)
    T = 40 * geo["dt"]

    def final(nsteps):
        w = np.zeros(nsteps + 1)
        _, m, _, _ = O.micro_solve(mi, af, geo["dx"], T / nsteps, nsteps, cfg.alpha_micro, Wd, w, 4, trace=True)
        return m

    ref = final(40 * 32)
    errs = [np.abs(final(40 * s) - ref).max() for s in (1, 2, 4)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8) and np.all(rates < 2.3), (errs, rates)


def _physics_1d(eps, points):
    K, mup, mu, eta = 20, 8.0, 3.9, 1.0
    cfg = W.config("c1_1d", eps=eps, pts_per_eps=K, box_n=int(2 * mup * K) + 1, mu_over_eps=mu)
    dt = O.micro_dt(cfg, eps / K)
    cfg = cfg.replace(micro_steps=int(np.ceil(eta * eps * eps / dt)))
    M0 = W.initial_field(cfg)
    H = O.micro_batch(cfg, M0, points=points)
    errs = []
    for j, p in enumerate(points):
        _, _, Q2 = O.q_derivatives_at_centre(cfg, M0, p)
        tgt = O.homogenised_target(np.array([[np.sqrt(0.75)]]), Q2)
        errs.append(np.linalg.norm(H[:, j] - tgt) / np.linalg.norm(tgt))
    return max(errs)


def test_physics_1d_harmonic_mean():
    """a = 1 + 0.5 sin(2 pi y): A^H = (int 1/a)^-1 = sqrt(3)/2 (EX1). E_avg ~ 1e-3 here."""
    assert _physics_1d(1 / 100, [0, 5, 17, 40]) < 5e-3


def test_physics_2d_separable_closed_form():
    """(EX3) coefficient: A^H = 1.1 sqrt(1.1^2 - 0.25) I; (EX2) initial data."""
    terms = [W._term(0.55, W._sin(0)), W._term(0.55, W._sin(1)), W._term(0.25, W._sin(0), W._sin(1))]
    eps, K = 1 / 400, 8
    cfg = W.HMMConfig(dim=2, n_macro=(24, 24, 1), alpha=0.01, alpha_micro=1.0, c0=1.21, terms=terms,
                      eps=eps, box_n=97, pts_per_eps=K, micro_steps=10, mu_over_eps=4.2)
    dt = O.micro_dt(cfg, eps / K)
    cfg = cfg.replace(micro_steps=int(np.ceil(0.5 * eps * eps / dt)))
    X1, X2 = np.meshgrid(*W.macro_coords(cfg), indexing="ij")
    M0 = W.ex2_initial(X1, X2).reshape(3, -1)
    p = 7 * 24 + 3
    H = O.micro_batch(cfg, M0, points=[p])[:, 0]
    _, _, Q2 = O.q_derivatives_at_centre(cfg, M0, p)
    tgt = O.homogenised_target(1.1 * np.sqrt(0.96) * np.eye(2), Q2)
    assert np.linalg.norm(H - tgt) / np.linalg.norm(tgt) < 2e-2


def test_constant_macro_field_gives_zero():
    cfg = W.config("c2_2d", n_macro=(8, 8, 1), box_n=24, micro_steps=30)
    M0 = np.tile(np.array([0.6, 0.0, 0.8])[:, None], (1, 64))
    H = O.micro_batch(cfg, M0, points=[0, 9, 63])
    # m_init is constant up to rounding (~1e-16), amplified by a/dx^2 ~ 1e7 before averaging
    assert np.abs(H).max() < 1e-8


def test_rotation_equivariance():
    cfg = W.config("c2_2d", n_macro=(8, 8, 1), box_n=24, micro_steps=30)
    M0 = W.initial_field(cfg)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    R = R @ np.array([[1, 0, 0], [0, np.cos(0.3), -np.sin(0.3)], [0, np.sin(0.3), np.cos(0.3)]])
    pts = [0, 13, 40]
    H = O.micro_batch(cfg, M0, points=pts)
    HR = O.micro_batch(cfg, R @ M0, points=pts)
    np.testing.assert_allclose(HR, R @ H, rtol=1e-9, atol=1e-9 * np.abs(H).max())


def test_ll_rhs_hand_value():
    """f(e_z, e_x) = -e_z x e_x - alpha e_z x (e_z x e_x) = (alpha, -1, 0)."""
    f = O.ll_rhs(np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0]), 0.3)
    np.testing.assert_allclose(f, [0.3, -1.0, 0.0], atol=1e-15)


def test_stepper_stability_limits_textbook_values():
    """RK4's stability interval on the imaginary axis is 2 sqrt(2); on the negative
    real axis both polynomials exit the unit disc at their textbook real limits
    (2 for Heun, 2.785293563405... for RK4), approached here with alpha -> infinity."""
    assert abs(O.stability_limit(1e-9, 1) - 2.0 * np.sqrt(2.0)) < 1e-6
    a = 1e4
    assert abs(O.stability_limit(a, 1) * abs(complex(-a, 1.0)) - 2.785293563405282) < 1e-4
    assert abs(O.stability_limit(a, 0) * abs(complex(-a, 1.0)) - 2.0) < 1e-4
    # HeunP's limit vanishes on the imaginary axis, RK4P's does not (Section 3.2)
    assert O.stability_limit(1e-4, 0) < 0.1 and O.stability_limit(1e-4, 1) > 2.8


def test_rk4p_fourth_order_in_time():
    cfg = W.config("c1_1d", n_macro=(16, 1, 1), box_n=41, micro_steps=10)
    M0 = W.initial_field(cfg)
    geo, mi, af, Wd, _ = _one_box(cfg, 5, M0)
    T = 40 * geo["dt"]

    def final(nsteps, stepper=1):
        w = np.zeros(nsteps + 1)
        _, m, _, _ = O.micro_solve(mi, af, geo["dx"], T / nsteps, nsteps, cfg.alpha_micro, Wd, w, 4,
                                   trace=True, stepper=stepper)
        return m

    ref = final(40 * 32)
    errs = [np.abs(final(40 * s) - ref).max() for s in (1, 2, 4)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.6) and np.all(rates < 4.4), (errs, rates)
    # HeunP and RK4P approximate the same solution
    assert np.abs(final(40 * 8, stepper=0) - ref).max() < 1e-3 * np.abs(ref - mi).max()


def test_rk4p_micro_batch_close_to_heunp():
    """At the same micro time and a small step, the two steppers give the same average."""
    cfg = W.config("c1_1d", n_macro=(16, 1, 1), box_n=81, micro_steps=240, dt_safety=0.2)
    M0 = W.initial_field(cfg)
    H0 = O.micro_batch(cfg, M0, points=[3, 9])
    dt0 = O.micro_dt(cfg, cfg.eps / cfg.pts_per_eps)
    cfg1 = cfg.replace(micro_stepper=1)
    dt1 = O.micro_dt(cfg1, cfg.eps / cfg.pts_per_eps)
    cfg1 = cfg1.replace(micro_steps=int(round(240 * dt0 / dt1)))
    cfg1 = cfg1.replace(dt_safety=cfg.dt_safety * dt0 * 240 / (cfg1.micro_steps * dt1))
    H1 = O.micro_batch(cfg1, M0, points=[3, 9])
    assert np.abs(H1 - H0).max() < 1e-3 * np.abs(H0).max(), (H0, H1)


def _ex2_error(inv_eps, mu_over_eps, K=8, mup=12.0, eta=2.0):
    """Relative E_avg of the (EX2) micro problem at one macro point, alpha_micro = 1,
    against A^H from the cell problem; mu', eta in units of eps and eps^2. Each
    distinct problem is solved once per test session."""
    return _ex2_error_cached(int(inv_eps), float(mu_over_eps), int(K), float(mup), float(eta))


@functools.lru_cache(maxsize=None)
def _ex2_error_cached(inv_eps, mu_over_eps, K, mup, eta):
    tp = 2 * np.pi

    def a(y1, y2):
        return (0.5 + (0.5 + 0.25 * np.sin(tp * y1)) * (0.5 + 0.25 * np.sin(tp * y2))
                + 0.25 * (np.cos(tp * (y1 - y2)) + np.sin(tp * y1)))

    AH = C.homogenised_coefficient_2d(a, 64)
    # the (EX2) coefficient as sums of separable products of the fast variable:
    # 0.75 + 0.375 sin y1 + 0.125 sin y2 + 0.3125 sin y1 sin y2 + 0.25 cos y1 cos y2
    terms = [W._term(0.375, W._sin(0)), W._term(0.125, W._sin(1)), W._term(0.3125, W._sin(0), W._sin(1)),
             W._term(0.25, W._cos(0), W._cos(1))]
    y = np.random.default_rng(5).random((2, 64))
    expanded = (0.75 + 0.375 * np.sin(tp * y[0]) + 0.125 * np.sin(tp * y[1])
                + 0.3125 * np.sin(tp * y[0]) * np.sin(tp * y[1]) + 0.25 * np.cos(tp * y[0]) * np.cos(tp * y[1]))
    np.testing.assert_allclose(expanded, a(y[0], y[1]), atol=1e-15)
    eps = 1.0 / inv_eps
    cfg = W.HMMConfig(dim=2, n_macro=(24, 24, 1), alpha=0.01, alpha_micro=1.0, c0=0.75, terms=terms, eps=eps,
                      box_n=int(round(2 * mup * K)) + 1, pts_per_eps=K, micro_steps=10, mu_over_eps=mu_over_eps)
    dt = O.micro_dt(cfg, eps / K)
    cfg = cfg.replace(micro_steps=int(np.ceil(eta * eps * eps / dt)))
    X1, X2 = np.meshgrid(*W.macro_coords(cfg), indexing="ij")
    M0 = W.ex2_initial(X1, X2).reshape(3, -1)
    p = 7 * 24 + 3
    H = O.micro_batch(cfg, M0, points=[p])[:, 0]
    _, _, Q2 = O.q_derivatives_at_centre(cfg, M0, p)
    tgt = O.homogenised_target(AH, Q2)
    return np.linalg.norm(H - tgt) / np.linalg.norm(tgt)


def test_ex2_error_falls_as_eps_squared():
    """(EX2) with alpha_micro = 1: E_avg at eps = 1/50 over E_avg at eps = 1/100.

    Section 4.4 compares the saturated errors of (EX2) for alpha = 1 at two values of
    eps a factor two apart and finds them a factor of about four apart. Here mu = 3.9
    eps (the section's averaging width), mu' = 12 eps and eta = 2 eps^2 are large
    enough that E_mu, E_mu' and E_eta are below E_eps (raising mu' to 14 eps or eta to
    2.5 eps^2 changes neither error by more than 15 %), and 8 points per eps with the
    order-4 stencil keep the discretisation error near 6e-6; the grids of the two
    boxes are identical in units of eps, so only the scale separation differs.
    """
    err = {inv_eps: _ex2_error(inv_eps, 3.9) for inv_eps in (50, 100)}
    assert err[50] < 5e-4 and err[100] < 2e-4, err
    assert 3.2 < err[50] / err[100] < 5.0, err


def test_ex2_error_against_averaging_width():
    """(EX2), eps = 1/100: E_avg against the averaging half-width mu (Section 4.4,
    averaging domain size). The bound E_mu <= C (mu^(px+1) + (eps/mu)^(qx+2)) with
    qx = 7 makes the error fall steeply while mu is a few eps, and the section finds
    it flat once mu is about 3.5 eps (the other terms then dominate): measured 2.4e-3
    at mu = 2 eps, 5.0e-5 at 3.5 eps, 5.3e-5 at 3.9 eps (the width of the eps pin above,
    whose value is reused) and 5.3e-5 at 4.5 eps; the pin is the fall to that level.
    """
    e2, e39 = (_ex2_error(100, mu) for mu in (2.0, 3.9))
    assert e2 > 20 * e39, (e2, e39)
    assert e39 < 1e-4


def test_ex2_error_against_averaging_time():
    """(EX2), eps = 1/100, mu = 3.9 eps, mu' = 10 eps: E_avg against the length eta of the
    time average (Section 4.4, length of the time interval eta). The bound
    E_eta <= C (eta^(pt+1) + (eps^2/eta)^(qt+1)) with qt = 7 makes the error fall
    steeply as eta grows through a few eps^2, faster for alpha = 1 than for small
    damping: measured 2.2e-2, 8.6e-4 and 7.7e-5 at eta = 0.5, 1 and 1.5 eps^2.
    """
    e05, e10, e15 = (_ex2_error(100, 3.9, 8, 10.0, eta) for eta in (0.5, 1.0, 1.5))
    assert e05 > 10 * e10 and e10 > 5 * e15, (e05, e10, e15)
    assert e15 < 2e-4


def test_ex2_error_against_box_size():
    """(EX2), eps = 1/100, mu = 3.9 eps, eta = 2 eps^2: E_avg against the half-width mu'
    of the computational box (Section 4.4, full domain size): with mu' only a little
    above mu the boundary error dominates, and it falls as mu' grows until the other
    terms remain: measured 2.1e-2, 2.2e-3, 1.3e-4, 5.3e-5 and 5.3e-5 at mu' = 6, 8, 10,
    12 and 14 eps (the paper has no model for this term; the pin is the fall).
    """
    e6, e8, e12 = (_ex2_error(100, 3.9, 8, mup, 2.0) for mup in (6.0, 8.0, 12.0))
    assert e6 > 5 * e8 > 5 * 5 * e12, (e6, e8, e12)
