"""Pins of the direct-simulation oracle (Section 5's reference solver: eq. prob
on a periodic grid resolving eps, conservative staggered stencil, MPEA).

What fixes each part independently of the oracle's own code:
* stencil: the discrete symbol of a single Fourier mode (closed form, order 2
  and 4, per axis), the Dirichlet-box stencil of the micro problems on the
  interior of a periodically padded copy, and H = -(1/dx^d) grad E_h by
  finite differences of the energy;
* time step: the AB3 stability limit on the imaginary axis (0.7236...) and the
  boundary-locus crossing for damped rays;
* time stepping: a precessing and damped spin wave, an exact solution of the
  semi-discrete equation for constant a, reached at second order in dt;
  |m| = 1 to rounding; monotone energy decay for alpha > 0;
* the patch evaluation used for sampled full-size parity equals the whole-grid
  run, including points whose patch wraps around the domain.
"""
import numpy as np
import pytest

import workloads as W
from oracle import dns_oracle as D
from oracle import hmm_oracle as O


def _const_cfg(n, a=1.3, alpha=0.0, order=4, dim=None):
    dim = len(n) if dim is None else dim
    return W.DNSConfig(dim=dim, n=tuple(n) + (1,) * (3 - len(n)), alpha=alpha, c0=a, terms=[],
                       eps=0.01, stencil_order=order)


def _var_cfg(n, alpha=0.1, order=4):
    cfg = W.dns_config("dns_quasi2d" if len(n) == 2 else "dns_loc1d")
    return cfg.replace(n=tuple(n) + (1,) * (3 - len(n)), alpha=alpha, stencil_order=order, eps=0.01)


def _sigma(theta, order):
    if order == 2:
        return 4.0 * np.sin(theta / 2) ** 2
    return ((27.0 * np.sin(theta / 2) - np.sin(1.5 * theta)) / 12.0) ** 2


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("n,k", [((24,), (3,)), ((20, 12), (2, 5)), ((9, 16), (4, 1))])
def test_fourier_symbol(order, n, k):
    cfg = _const_cfg(n, a=1.7, order=order)
    X = np.meshgrid(*[np.arange(v) / v for v in n], indexing="ij")
    ph = 2 * np.pi * sum(kk * x for kk, x in zip(k, X))
    m = np.stack([np.cos(ph), np.sin(ph), np.full_like(ph, 0.3)])
    H = D.field_H(m, D.face_coefficients(cfg), D.grid_spacing(cfg), order)
    lam = 1.7 * sum(_sigma(2 * np.pi * kk / v, order) * v * v for kk, v in zip(k, n))
    np.testing.assert_allclose(H[0], -lam * m[0], atol=1e-9 * lam)
    np.testing.assert_allclose(H[1], -lam * m[1], atol=1e-9 * lam)
    np.testing.assert_allclose(H[2], 0.0, atol=1e-9 * lam)


@pytest.mark.parametrize("order", [2, 4])
def test_matches_dirichlet_stencil_on_padded_copy(order):
    cfg = _var_cfg((13, 13), order=order)    # the box stencil takes cubic boxes
    r = 1 if order == 2 else 3
    m = W.dns_initial(cfg, noise=0.3).reshape((3,) + cfg.shape)
    H = D.field_H(m, D.face_coefficients(cfg), D.grid_spacing(cfg), order)
    idx = [np.arange(-r, v + r) for v in cfg.shape]
    mp = m[np.ix_(range(3), *[i % v for i, v in zip(idx, cfg.shape)])]
    # faces j + 1/2 of the padded array, j = 0..len-2, at their true positions
    af = [a[tuple(slice(0, a.shape[ax] - 1) if ax == k else slice(None) for ax in range(2))]
          for k, a in enumerate(D.face_coefficients(cfg, idx))]
    Hd = O.field_H(mp, af, D.grid_spacing(cfg)[0], order)
    np.testing.assert_allclose(Hd, H, rtol=0, atol=1e-10 * np.abs(H).max())


@pytest.mark.parametrize("order", [2, 4])
def test_energy_gradient(order):
    cfg = _var_cfg((9, 7), order=order)
    shape = (3,) + cfg.shape
    dx = D.grid_spacing(cfg)
    af = D.face_coefficients(cfg)
    m = W.dns_initial(cfg, noise=0.2).reshape(shape)
    H = D.field_H(m, af, dx, order)
    vol = np.prod(dx)
    h = 1e-6
    for c, i, j in [(0, 0, 0), (1, 4, 3), (2, 8, 6), (0, 5, 1)]:
        mp, mm = m.copy(), m.copy()
        mp[c, i, j] += h
        mm[c, i, j] -= h
        g = (D.exchange_energy(mp, af, dx, order) - D.exchange_energy(mm, af, dx, order)) / (2 * h)
        assert abs(-g / vol - H[c, i, j]) < 1e-6 * np.abs(H).max()


def test_ab3_limit_imaginary_axis():
    # AB3's stability interval on the imaginary axis is [-0.7236i, 0.7236i]
    assert abs(D.ab3_stability_limit(0.0) - 0.7236) < 1e-4


@pytest.mark.parametrize("alpha", [0.0, 0.01, 0.1, 1.0])
def test_ab3_limit_on_boundary_locus(alpha):
    """The limit s(-alpha + i) lies on the boundary locus z(theta) =
    12 (zeta^3 - zeta^2)/(23 zeta^2 - 16 zeta + 5), zeta = e^{i theta}: the
    first crossing of the ray by the locus, found here by bisection on theta."""
    s = D.ab3_stability_limit(alpha)
    w = complex(-alpha, 1.0)

    def z(t):
        q = np.exp(1j * t)
        return 12 * (q ** 3 - q ** 2) / (23 * q ** 2 - 16 * q + 5)

    def off_ray(t):                       # signed distance of z(t) from the ray's line
        v = z(t)
        return (v * np.conj(w)).imag

    ts = np.linspace(1e-4, np.pi, 20001)
    f = np.array([off_ray(t) for t in ts])
    crossings = []
    for i in np.nonzero(np.sign(f[1:]) != np.sign(f[:-1]))[0]:
        lo, hi = ts[i], ts[i + 1]
        for _ in range(80):
            mid = 0.5 * (lo + hi)
            if np.sign(off_ray(mid)) == np.sign(off_ray(lo)):
                lo = mid
            else:
                hi = mid
        v = z(lo)
        if (v * np.conj(w)).real > 0:     # on the ray, not its opposite
            crossings.append(abs(v) / abs(w))
    assert crossings
    assert abs(min(crossings) - s) < 1e-6 * s


def _spin_wave(cfg, k, theta0, t):
    """Semi-discrete exact solution for constant a: m = (s cos phi, s sin phi, c)."""
    n = cfg.shape
    X = np.meshgrid(*[np.arange(v) / v for v in n], indexing="ij")
    ph0 = 2 * np.pi * sum(kk * x for kk, x in zip(k, X))
    lam = cfg.c0 * sum(_sigma(2 * np.pi * kk / v, cfg.stencil_order) * v * v for kk, v in zip(k, n))
    if cfg.alpha == 0:
        th, ph = theta0, ph0 + lam * np.cos(theta0) * t
    else:
        T0 = np.tan(theta0)
        kap = cfg.alpha * lam
        th = np.arctan(T0 * np.exp(-kap * t))
        ph = ph0 + (np.arcsinh(np.exp(kap * t) / T0) - np.arcsinh(1.0 / T0)) / cfg.alpha
    th = np.broadcast_to(th, ph0.shape)
    return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)]).reshape(3, -1)


@pytest.mark.parametrize("alpha", [0.0, 0.3])
@pytest.mark.parametrize("n,k", [((32,), (2,)), ((16, 12), (1, 2))])
def test_spin_wave_second_order(alpha, n, k):
    cfg = _const_cfg(n, a=1.3, alpha=alpha)
    dt0 = D.dns_dt(cfg)
    T = 48 * dt0
    errs = []
    for f in (4, 8, 16):                  # the asymptotic range (dt0: the default step)
        run = D.DNS(cfg, _spin_wave(cfg, k, 0.8, 0.0), dt=dt0 / f)
        run.step(48 * f)
        errs.append(np.abs(run.M - _spin_wave(cfg, k, 0.8, T)).max())
    assert errs[2] < 1e-7
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert r1 > 3.4 and r2 > 3.4, errs


def test_norm_and_energy_decay():
    cfg = _var_cfg((12, 10), alpha=0.1)
    run = D.DNS(cfg, W.dns_initial(cfg, noise=0.2))
    E = [run.energy()]
    for _ in range(25):
        run.step()
        E.append(run.energy())
        assert np.abs(np.sqrt((run.M ** 2).sum(0)) - 1).max() < 1e-13
    assert all(b < a for a, b in zip(E, E[1:])), E


@pytest.mark.parametrize("order", [2, 4])
def test_patch_run_equals_whole_grid(order):
    cfg = _var_cfg((40, 36), alpha=0.05, order=order)
    M0 = W.dns_initial(cfg, noise=0.1)
    dt = D.dns_dt(cfg)
    run = D.DNS(cfg, M0, dt=dt)
    run.step(4)
    M = run.M.reshape((3,) + cfg.shape)
    for c in [(0, 0), (20, 17), (39, 2), (5, 35)]:
        v = D.patch_run(cfg, M0, c, 4, dt)
        np.testing.assert_allclose(v, M[:, c[0], c[1]], rtol=0, atol=1e-14)


def test_named_configs():
    q = W.dns_config("dns_quasi2d")
    X = np.meshgrid(*W.dns_coords(q.replace(n=(50, 40, 1))), indexing="ij")
    a = O.coef_eval(q, q.eps, X)
    tp = 2 * np.pi
    ref = (1 + 0.25 * np.sin(tp * X[0] / 0.01)) * (1 + 0.25 * np.sin(tp * X[1] / 0.01)
                                                   + 0.25 * np.sin(tp * 1.41 * X[1] / 0.01))
    np.testing.assert_allclose(a, ref, rtol=1e-12)
    l1 = W.dns_config("dns_loc1d")
    x = np.linspace(0, 1, 777)
    ref = 1.1 + 0.25 * np.sin(tp * x + 1.1) + 0.5 * np.sin(tp * x * 400)
    np.testing.assert_allclose(O.coef_eval(l1, l1.eps, [x]), ref, rtol=1e-11)
    assert l1.n_points == 6000 and q.n_points == 1500 ** 2
