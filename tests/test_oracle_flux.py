"""Pins of the flux-model oracle (Section 2.2, eq. macro_flux).

* F_avg -> A^H grad m: in 1D with a = 1 + 0.5 sin(2 pi y) (A^H = sqrt(3)/2, the
  harmonic mean, EX1's coefficient) the averaged flux at the staggered point
  x_i + DX/2 matches a_H m0'(x_i + DX/2) of the exact macro data, and the flux
  model's field div F_avg matches a_H m0''(x_i) on every macro point; the
  derivatives are of the closed-form initial data, not of anything the
  oracle computes.
* The macro divergence reproduces the closed-form symbol of the staggered
  difference on a Fourier mode (orders 2 and 4, per axis).
* Constant macro data gives zero flux; rotating M rotates F.
* The 2D separable (EX3) coefficient: F_avg -> A^H grad m with A^H = 1.1 sqrt(0.96) I.
"""
import numpy as np
import pytest

import workloads as W
from oracle import flux_oracle as F
from oracle import hmm_oracle as O

AH1 = np.sqrt(0.75)


def _m0(x):
    mt = np.stack([0.5 + 0.3 * np.sin(2 * np.pi * x), 0.4 * np.cos(2 * np.pi * x), 0.6 + 0 * x])
    return mt / np.sqrt((mt ** 2).sum(0))


def _d(f, x, h):
    return (f(x + h) - f(x - h)) / (2 * h)


def _cfg_1d(n_macro=64, eps=1 / 100):
    K, mup, mu, eta = 20, 8.0, 3.9, 1.0
    cfg = W.config("c1_1d", n_macro=(n_macro, 1, 1), eps=eps, pts_per_eps=K,
                   box_n=int(2 * mup * K) + 1, mu_over_eps=mu)
    dt = O.micro_dt(cfg, eps / K)
    return cfg.replace(micro_steps=int(np.ceil(eta * eps * eps / dt)))


def test_flux_1d_harmonic_mean():
    cfg = _cfg_1d()
    M0 = W.initial_field(cfg)
    pts = [0, 5, 17, 40]
    Fl = F.micro_batch_flux(cfg, M0, points=pts)
    for j, p in enumerate(pts):
        x = np.array([(p + 0.5) / 64])
        tgt = AH1 * _d(_m0, x, 1e-5)[:, 0]
        assert np.linalg.norm(Fl[0, :, j] - tgt) / np.linalg.norm(tgt) < 5e-4, p


def test_flux_field_1d_second_derivative():
    """div F_avg -> a_H m0'' with the staggered difference's fourth order in DX."""
    errs = []
    for n in (16, 32):
        cfg = _cfg_1d(n_macro=n)
        x = np.arange(n) / n
        M0 = W.c1_initial(x)
        H = F.flux_field(cfg, M0)
        tgt = AH1 * (_m0(x + 1e-4) - 2 * _m0(x) + _m0(x - 1e-4)) / 1e-8
        errs.append(np.linalg.norm(H - tgt, axis=0).max() / np.linalg.norm(tgt, axis=0).max())
        if n == 32:
            # the field model's H_avg approximates the same quantity
            Hf = O.micro_batch(cfg, M0, points=[0, 7])
            assert np.linalg.norm(Hf - H[:, [0, 7]], axis=0).max() / np.linalg.norm(tgt, axis=0).max() < 5e-3
    # a second-order divergence would give a ratio of 4 (the upscaling error, ~1e-4 here, caps it)
    assert errs[1] < 2e-3 and errs[0] / errs[1] > 6, errs


@pytest.mark.parametrize("order", [2, 4])
def test_divergence_symbol(order):
    cfg = W.config("c2_2d", n_macro=(12, 20, 1), interp_order=order)
    n = (12, 20)
    X = np.meshgrid(np.arange(n[0]) / n[0], np.arange(n[1]) / n[1], indexing="ij")
    kap = (2, 3)
    Fx = np.zeros((2, 3) + n)
    # column k sampled at the staggered points x_i + (DX_k / 2) e_k
    for k in range(2):
        Xs = [X[a] + (0.5 / n[a] if a == k else 0.0) for a in range(2)]
        ph = 2 * np.pi * (kap[0] * Xs[0] + kap[1] * Xs[1])
        Fx[k, 0] = np.sin(ph)
        Fx[k, 1] = np.cos(ph)
        Fx[k, 2] = 0.3
    div = F.flux_divergence(cfg, Fx.reshape(2, 3, -1)).reshape((3,) + n)
    ph = 2 * np.pi * (kap[0] * X[0] + kap[1] * X[1])
    lam = 0.0
    for k in range(2):
        th = 2 * np.pi * kap[k] / n[k]
        g = 2 * np.sin(th / 2) if order == 2 else (27 * np.sin(th / 2) - np.sin(1.5 * th)) / 12
        lam += g * n[k]
    np.testing.assert_allclose(div[0], lam * np.cos(ph), atol=1e-10 * lam)
    np.testing.assert_allclose(div[1], -lam * np.sin(ph), atol=1e-10 * lam)
    np.testing.assert_allclose(div[2], 0.0, atol=1e-10 * lam)


def test_constant_macro_field_gives_zero_flux():
    cfg = W.config("c2_2d", n_macro=(8, 8, 1), box_n=24, micro_steps=30, interp_order=4)
    M0 = np.tile(np.array([0.6, 0.0, 0.8])[:, None], (1, 64))
    Fl = F.micro_batch_flux(cfg, M0, points=[0, 9, 63])
    assert np.abs(Fl).max() < 1e-9


def test_rotation_equivariance():
    cfg = W.config("c2_2d", n_macro=(8, 8, 1), box_n=24, micro_steps=30)
    M0 = W.initial_field(cfg)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0.0], [np.sin(th), np.cos(th), 0.0], [0.0, 0.0, 1.0]])
    R = R @ np.array([[1.0, 0.0, 0.0], [0.0, np.cos(0.4), -np.sin(0.4)], [0.0, np.sin(0.4), np.cos(0.4)]])
    pts = [3, 40]
    A = F.micro_batch_flux(cfg, M0, points=pts)
    B = F.micro_batch_flux(cfg, R @ M0, points=pts)
    for k in range(2):
        np.testing.assert_allclose(B[k], R @ A[k], atol=1e-9 * np.abs(A).max())


def test_flux_2d_separable_closed_form():
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
    i0, i1 = divmod(p, 24)
    Fl = F.micro_batch_flux(cfg, M0, points=[p])
    aH = 1.1 * np.sqrt(0.96)
    for k in range(2):
        x = [i0 / 24 + (0.5 / 24 if k == 0 else 0.0), i1 / 24 + (0.5 / 24 if k == 1 else 0.0)]
        h = 1e-5
        xp, xm = list(x), list(x)
        xp[k] += h
        xm[k] -= h
        grad = (W.ex2_initial(np.array(xp[0]), np.array(xp[1])) - W.ex2_initial(np.array(xm[0]), np.array(xm[1]))) / (2 * h)
        tgt = aH * np.asarray(grad).reshape(3)
        assert np.linalg.norm(Fl[k, :, 0] - tgt) / np.linalg.norm(tgt) < 2e-2, k
