"""Pins of the oracle's smoothing kernels and quadrature weights.

The kernel spaces K^{p,q} and K0^{p,q} are fixed by Section 2.3 (Definition of
smoothing kernels): compact support, q continuous derivatives, unit mass and p
vanishing moments. These are checked by Gauss-Legendre quadrature and by
numpy's polynomial algebra, routes independent of the oracle's rational solve.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import Polynomial

from oracle import hmm_oracle as O


def _gauss(a, b, n=80):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


@pytest.mark.parametrize("p,q", [(3, 7), (1, 3), (5, 9)])
def test_space_kernel_moments(p, q):
    x, w = _gauss(-1.0, 1.0)
    K = O.kernel_eval(x, p, q)
    for r in range(p + 1):
        mom = np.sum(w * K * x ** r)
        assert abs(mom - (1.0 if r == 0 else 0.0)) < 1e-12, (r, mom)
    # the next even moment must not vanish (p moments exactly, not more)
    r = p + 1 if (p + 1) % 2 == 0 else p + 2
    assert abs(np.sum(w * K * x ** r)) > 1e-6


@pytest.mark.parametrize("p,q", [(3, 7), (1, 3), (2, 5)])
def test_time_kernel_moments(p, q):
    t, w = _gauss(0.0, 1.0)
    K0 = O.kernel0_eval(t, p, q)
    for r in range(p + 1):
        mom = np.sum(w * K0 * t ** r)
        assert abs(mom - (1.0 if r == 0 else 0.0)) < 1e-9 * max(1.0, np.abs(K0).max()), (r, mom)
    assert np.all(O.kernel0_eval(np.array([-0.5, -1e-9, 0.0, 1.0, 1.3]), p, q) == 0.0)


@pytest.mark.parametrize("p,q", [(3, 7), (1, 3)])
def test_kernel_smoothness_at_support_ends(p, q):
    """K in C_c^q: derivatives 0..q vanish at +-1 (K0: at 0 and 1); the (q+1)-th does not."""
    c = [float(v) for v in O.kernel_coefficients(p, q)]
    K = Polynomial([1.0, 0.0, -1.0]) ** (q + 1) * Polynomial(c)
    for x0 in (-1.0, 1.0):
        for j in range(q + 1):
            assert abs(K.deriv(j)(x0)) < 1e-7 * (1 + abs(K.deriv(j).coef).max())
        assert abs(K.deriv(q + 1)(x0)) > 1e-3
    c0 = [float(v) for v in O.kernel0_coefficients(p, q)]
    K0 = (Polynomial([0.0, 1.0]) * Polynomial([1.0, -1.0])) ** (q + 1) * Polynomial(c0)
    for t0 in (0.0, 1.0):
        for j in range(q + 1):
            assert abs(K0.deriv(j)(t0)) < 1e-6 * (1 + abs(K0.deriv(j).coef).max())
    # the evaluator agrees with the polynomial algebra inside the support
    xs = np.linspace(-0.99, 0.99, 41)
    np.testing.assert_allclose(O.kernel_eval(xs, p, q), K(xs), rtol=1e-10, atol=1e-12)
    ts = np.linspace(0.01, 0.99, 41)
    # the expanded polynomial has coefficients ~1e10: compare on the scale of max|K0|
    np.testing.assert_allclose(O.kernel0_eval(ts, p, q), K0(ts), rtol=0, atol=1e-6 * np.abs(K0(ts)).max())


def test_space_kernel_is_even_and_compact():
    x = np.linspace(-1.5, 1.5, 301)
    K = O.kernel_eval(x)
    np.testing.assert_allclose(K, O.kernel_eval(-x), rtol=1e-14, atol=1e-16)
    assert np.all(K[np.abs(x) >= 1.0] == 0.0)


@pytest.mark.parametrize("N,K", [(64, 8.0), (201, 20.0), (97, 8.0)])
def test_discrete_space_weights(N, K):
    eps = 1.0 / 200
    dx = eps / K
    mu = 0.8 * (N - 1) * dx / 2
    W = O.space_weights(N, dx, mu, 3, 7)
    xi = (np.arange(N) - (N - 1) / 2) * dx
    assert abs(W.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(W, W[::-1], atol=1e-17)
    assert np.all(W[np.abs(xi) >= mu] == 0.0)
    # trapezoid rule on a C^7 kernel: moments 1..3 vanish to quadrature accuracy
    for r in (1, 2, 3):
        assert abs(np.sum(W * (xi / mu) ** r)) < 1e-9


def test_discrete_time_weights():
    M = 400
    w = O.time_weights(M, 3, 7)
    t = np.arange(M + 1) / M
    assert w[0] == 0.0 and w[-1] == 0.0
    assert abs(w.sum() - 1.0) < 1e-14
    for r in (1, 2, 3):
        assert abs(np.sum(w * t ** r)) < 1e-9


def test_heun_stability_limit_matches_cubic():
    """|R(s w)|^2 = 1 with R = 1 + z + z^2/2, w = -alpha + i, reduces to the cubic
    (1+a^2)^2/4 s^3 - a(1+a^2) s^2 + 2 a^2 s - 2a = 0; its smallest positive root is the limit."""
    for a in (0.01, 0.1, 0.5, 1.0, 1.2, 2.0):
        roots = np.roots([(1 + a * a) ** 2 / 4, -a * (1 + a * a), 2 * a * a, -2 * a])
        pos = sorted(r.real for r in roots if abs(r.imag) < 1e-12 and r.real > 0)
        assert abs(O.heun_stability_limit(a) - pos[0]) < 1e-9, a


def test_heun_stability_limit_small_alpha_asymptote():
    # for alpha -> 0 the cubic gives s^3/4 ~ 2 alpha: Heun does not contain the imaginary axis
    a = 1e-5
    assert abs(O.heun_stability_limit(a) / (8 * a) ** (1 / 3) - 1.0) < 2e-2


def test_stencil_symbol_max_matches_dense_eigenvalues():
    """The largest eigenvalue of -D_s D_s on a long periodic line is lambda_s/dx^2."""
    for order in (2, 4):
        n = 256
        if order == 2:
            c = {-1: 1.0, 0: -2.0, 1: 1.0}
        else:
            # node i from faces i+jj+1/2, jj = -2..1; face j+1/2 from nodes j-1..j+2
            hh = {-2: 1 / 24, -1: -27 / 24, 0: 27 / 24, 1: -1 / 24}
            g = {-1: 1 / 24, 0: -27 / 24, 1: 27 / 24, 2: -1 / 24}
            c = {}
            for jj, vh in hh.items():
                for a, vg in g.items():
                    c[jj + a] = c.get(jj + a, 0.0) + vh * vg
        A = np.zeros((n, n))
        for i in range(n):
            for off, v in c.items():
                A[i, (i + off) % n] += v
        lam = np.linalg.eigvalsh(-0.5 * (A + A.T)).max()
        assert abs(lam - O.stencil_symbol_max(order)) < 1e-9
