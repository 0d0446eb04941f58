"""Pins of the oracle's H = div(a^eps grad m) stencil (Section 2.3; 4th order per the configs).

* Manufactured smooth m and a: the error against the analytic div(a grad m)
  falls as dx^2 (order 2) and dx^4 (order 4), in 1D, 2D and 3D.
* H = -(1/dx^d) dE_h/dm at interior nodes (the discrete energy identity that
  makes the micro dynamics dissipative for alpha > 0).
* Constant fields give H = 0; the operator is symmetric on fields vanishing on the ring.
"""
import numpy as np
import pytest
import sympy as sy

from oracle import hmm_oracle as O

xs = sy.symbols("x1 x2 x3", real=True)


def _manufactured(d):
    x = xs[:d]
    a = 1 + sy.Rational(3, 10) * sy.sin(2 * sy.pi * x[0] + 0.4)
    if d > 1:
        a = a * (1 + sy.Rational(1, 4) * sy.cos(2 * sy.pi * x[1]))
    if d > 2:
        a = a + sy.Rational(1, 5) * sy.sin(2 * sy.pi * (x[2] - x[0]))
    m = [sy.sin(2 * sy.pi * x[0]) + sum(sy.cos(2 * sy.pi * (k + 1) * x[k]) for k in range(1, d)),
         sy.cos(4 * sy.pi * x[0] + 0.3) * (1 if d == 1 else sy.sin(2 * sy.pi * x[1])),
         sy.exp(sy.sin(2 * sy.pi * x[d - 1]))]
    H = [sum(sy.diff(a * sy.diff(mc, x[k]), x[k]) for k in range(d)) for mc in m]
    return (sy.lambdify(x, a, "numpy"), [sy.lambdify(x, mc, "numpy") for mc in m],
            [sy.lambdify(x, hc, "numpy") for hc in H])


def _grid_error(d, N, order):
    a_f, m_f, H_f = _manufactured(d)
    dx = 1.0 / (N - 1)
    nodes = np.arange(N) * dx
    faces = (np.arange(N - 1) + 0.5) * dx
    X = np.meshgrid(*([nodes] * d), indexing="ij")
    m = np.stack([np.broadcast_to(f(*X), X[0].shape) for f in m_f])
    af = []
    for k in range(d):
        c = [faces if a == k else nodes for a in range(d)]
        af.append(np.broadcast_to(a_f(*np.meshgrid(*c, indexing="ij")),
                                  tuple(N - 1 if a == k else N for a in range(d))).copy())
    H = O.field_H(m, af, dx, order)
    r = 1 if order == 2 else 3
    Xi = np.meshgrid(*([nodes[r:N - r]] * d), indexing="ij")
    Hex = np.stack([np.broadcast_to(f(*Xi), Xi[0].shape) for f in H_f])
    return np.abs(H - Hex).max()


@pytest.mark.parametrize("d,order,sizes,expect", [
    (1, 2, (33, 65, 129), 2.0), (1, 4, (33, 65, 129), 4.0),
    (2, 2, (25, 49, 97), 2.0), (2, 4, (25, 49, 97), 4.0),
    (3, 4, (13, 25, 49), 4.0),
])
def test_manufactured_order(d, order, sizes, expect):
    errs = [_grid_error(d, N, order) for N in sizes]
    # dx halves (nearly) between sizes
    hs = [1.0 / (N - 1) for N in sizes]
    slopes = [np.log(errs[i] / errs[i + 1]) / np.log(hs[i] / hs[i + 1]) for i in range(len(errs) - 1)]
    assert slopes[-1] > expect - 0.3, (errs, slopes)


@pytest.mark.parametrize("d,order", [(1, 4), (2, 2), (2, 4), (3, 4)])
def test_energy_identity(d, order):
    rng = np.random.default_rng(11 + d + order)
    N = 12 if d < 3 else 9
    dx = 0.37
    m = rng.standard_normal((3,) + (N,) * d)
    af = [0.5 + rng.random(tuple(N - 1 if a == k else N for a in range(d))) for k in range(d)]
    H = O.field_H(m, af, dx, order)
    r = 1 if order == 2 else 3
    for trial in range(6):
        idx = tuple(rng.integers(r, N - r, size=d))
        c = int(rng.integers(0, 3))
        step = 1e-3
        mp, mm = m.copy(), m.copy()
        mp[(c,) + idx] += step
        mm[(c,) + idx] -= step
        dE = (O.exchange_energy(mp, af, dx, order) - O.exchange_energy(mm, af, dx, order)) / (2 * step)
        Hp = H[(c,) + tuple(i - r for i in idx)]
        assert abs(-dE / dx ** d - Hp) < 1e-9 * (1 + abs(Hp)), (idx, c, -dE / dx ** d, Hp)


def test_constant_field_and_symmetry():
    rng = np.random.default_rng(5)
    N, d, order, dx = 14, 2, 4, 0.1
    af = [0.5 + rng.random((N - 1, N)), 0.5 + rng.random((N, N - 1))]
    const = np.ones((3, N, N)) * np.array([0.2, -0.4, 0.9])[:, None, None]
    assert np.abs(O.field_H(const, af, dx, order)).max() < 1e-12
    r = 3
    u = np.zeros((3, N, N))
    v = np.zeros((3, N, N))
    u[:, r:N - r, r:N - r] = rng.standard_normal((3, N - 2 * r, N - 2 * r))
    v[:, r:N - r, r:N - r] = rng.standard_normal((3, N - 2 * r, N - 2 * r))
    lhs = (u[:, r:N - r, r:N - r] * O.field_H(v, af, dx, order)).sum()
    rhs = (v[:, r:N - r, r:N - r] * O.field_H(u, af, dx, order)).sum()
    assert abs(lhs - rhs) < 1e-9 * abs(lhs)
    # negative semi-definite
    assert (u[:, r:N - r, r:N - r] * O.field_H(u, af, dx, order)).sum() < 0


def test_batched_equals_single():
    rng = np.random.default_rng(9)
    N, dx = 16, 0.2
    m = rng.standard_normal((4, 3, N, N))
    af = [0.5 + rng.random((4, N - 1, N)), 0.5 + rng.random((4, N, N - 1))]
    Hb = O.field_H(m, af, dx, 4)
    for b in range(4):
        np.testing.assert_allclose(Hb[b], O.field_H(m[b], [af[0][b], af[1][b]], dx, 4), rtol=1e-14)
