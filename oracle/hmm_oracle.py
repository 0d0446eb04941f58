"""Plain FP64 CPU oracle of the HMM micro-problem path and its macro step.

TEST INFRASTRUCTURE ONLY. This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by ``bench.py``'s CPU-baseline/reference leg,
and by nothing else. The product (the CUDA library and its Python binding)
never imports, links or executes anything under ``oracle/``; the two share no
code. Inputs come from the ``workloads`` module, which holds no arithmetic of
the method.

What it computes, following Leitenmaier & Runborg, "Heterogeneous multiscale
methods for the Landau-Lifshitz equation", step by step and in FP64:

* smoothing kernels K in K^{p,q} and K0 in K0^{p,q} (Section 2.3, Definition
  of smoothing kernels), built from exact rational moments;
* the kernel-weighted space-time average (Section 2.3, eq. upscaling),
  discretised by the trapezoid rule with weights normalised to sum 1;
* the micro initial data Q_[2k] = P_[2k]/|P_[2k]| (Section 4.1, eq. Q_k),
  interpolating one dimension after the other;
* the micro problem (Section 2.2, eq. micro) on [-mu', mu']^d with Dirichlet
  conditions on m - m_init (Section 4.2), H = div(a^eps grad m) by a
  conservative staggered difference (2nd order as in Section 2.3, or 4th order);
* HeunP, RK4P, MPE or MPEA micro time stepping (Section 3.1) with the micro
  time step bounded by the stability condition eq. Cstab (Section 3.2);
* the field-model macro step (Section 2.2, eq. macro_disc) by MPEA
  (Section 3.1, eqs. h_term, h_mpea, mpe_update) or MPE (eq. h_mpe) with an
  RK4P start-up.

Where the paper is silent or garbled, the reading taken is stated where it is
used and marked "a reading".
Every function here is pinned by the `-m "not gpu"` tests in tests/test_oracle_*.py.
"""
from __future__ import annotations

import math
from fractions import Fraction
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

# --------------------------------------------------------------------------
# Smoothing kernels (Section 2.3, Definition of K^{p,q} and K0^{p,q})
# --------------------------------------------------------------------------


def _binom(n: int, k: int) -> int:
    return math.comb(n, k)


def kernel_coefficients(p: int, q: int) -> List[Fraction]:
    """Coefficients c_0..c_p of K(x) = (1-x^2)^(q+1) * sum_k c_k x^k on [-1, 1].

    K vanishes with its first q derivatives at x = +-1, so K is in C_c^q([-1,1])
    and K^(q+1) is of bounded variation; the c_k are fixed by the p+1 moment
    conditions int K x^r dx = delta_{r0}, r = 0..p (a reading: the paper gives
    only the kernel space, not a formula). Solved exactly in rationals.
    """
    def base_moment(n: int) -> Fraction:
        # int_{-1}^{1} (1-x^2)^(q+1) x^n dx, expanded binomially
        tot = Fraction(0)
        for i in range(q + 2):
            e = 2 * i + n
            if e % 2 == 0:
                tot += Fraction((-1) ** i * _binom(q + 1, i) * 2, e + 1)
        return tot

    A = [[base_moment(k + r) for k in range(p + 1)] for r in range(p + 1)]
    b = [Fraction(1 if r == 0 else 0) for r in range(p + 1)]
    return _solve_fractions(A, b)


def kernel0_coefficients(p: int, q: int) -> List[Fraction]:
    """Coefficients d_0..d_p of K0(t) = t^(q+1) (1-t)^(q+1) sum_k d_k t^k on [0, 1].

    K0 is zero for t <= 0 (one-sided, K0 in K0^{p,q}), vanishes with its first
    q derivatives at t = 0 and t = 1, and has int K0 t^r dt = delta_{r0}, r = 0..p.
    """
    def base_moment(n: int) -> Fraction:
        # int_0^1 t^(q+1+n) (1-t)^(q+1) dt, expanded binomially
        tot = Fraction(0)
        for i in range(q + 2):
            tot += Fraction((-1) ** i * _binom(q + 1, i), q + 2 + n + i)
        return tot

    A = [[base_moment(k + r) for k in range(p + 1)] for r in range(p + 1)]
    b = [Fraction(1 if r == 0 else 0) for r in range(p + 1)]
    return _solve_fractions(A, b)


def _solve_fractions(A: List[List[Fraction]], b: List[Fraction]) -> List[Fraction]:
    n = len(b)
    M = [row[:] + [b[i]] for i, row in enumerate(A)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        for r in range(n):
            if r != col and M[r][col] != 0:
                fac = M[r][col] / M[col][col]
                M[r] = [x - fac * y for x, y in zip(M[r], M[col])]
    return [M[i][n] / M[i][i] for i in range(n)]


def _as(v: Fraction, dtype):
    """A rational in the working precision (numerator and denominator rounded once each)."""
    return dtype(v.numerator) / dtype(v.denominator)


def _pi(dtype):
    return dtype(np.pi) if np.dtype(dtype) == np.float64 else 4 * np.arctan(dtype(1))


def kernel_eval(x, p: int = 3, q: int = 7, dtype=np.float64) -> np.ndarray:
    """K(x) in K^{p,q}, zero outside (-1, 1)."""
    c = [_as(v, dtype) for v in kernel_coefficients(p, q)]
    x = np.asarray(x, dtype=dtype)
    poly = np.zeros_like(x)
    for k in reversed(range(len(c))):
        poly = poly * x + c[k]
    inside = np.abs(x) < 1.0
    return np.where(inside, (1.0 - x * x) ** (q + 1) * poly, 0.0)


def kernel0_eval(t, p: int = 3, q: int = 7, dtype=np.float64) -> np.ndarray:
    """K0(t) in K0^{p,q}, zero outside (0, 1)."""
    c = [_as(v, dtype) for v in kernel0_coefficients(p, q)]
    t = np.asarray(t, dtype=dtype)
    poly = np.zeros_like(t)
    for k in reversed(range(len(c))):
        poly = poly * t + c[k]
    inside = (t > 0.0) & (t < 1.0)
    return np.where(inside, (t * (1.0 - t)) ** (q + 1) * poly, 0.0)


def space_weights(N: int, dx: float, mu: float, p: int, q: int, dtype=np.float64) -> np.ndarray:
    """Discrete 1D weights of K_mu at the micro nodes xi_j (eq. upscaling).

    Trapezoid rule: W_j proportional to dx*K_mu(xi_j) = (dx/mu) K(xi_j/mu), then
    normalised to sum exactly 1 (a reading: the paper fixes no quadrature).
    xi_j = (j - (N-1)/2) dx: the box centred on its macro point.
    """
    xi = (np.arange(N, dtype=dtype) - dtype(N - 1) / 2) * dtype(dx)
    W = kernel_eval(xi / dtype(mu), p, q, dtype)
    return W / W.sum()


def time_weights(M: int, p: int, q: int, dtype=np.float64) -> np.ndarray:
    """Discrete weights w_n, n = 0..M, of K0_eta at t_n = n*dt, eta = M*dt.

    Trapezoid rule, normalised to sum exactly 1 (a reading: the paper fixes no
    quadrature). w_0 = w_M = 0.
    """
    t = np.arange(M + 1, dtype=dtype) / dtype(M)
    w = kernel0_eval(t, p, q, dtype)
    return w / w.sum()


# --------------------------------------------------------------------------
# Stability limit of HeunP on the eigenvalue ray (Section 3.2, eq. Cstab)
# --------------------------------------------------------------------------


HEUNP, RK4P, MICRO_MPE, MICRO_MPEA = 0, 1, 2, 3   # micro steppers (Section 3.1)


def _growth(stepper: int):
    """Growth factor of the stepper's linear stability analysis at z = lambda dt.

    HeunP (0) and RK4P (1): |R(z)| with R = 1 + z + z^2/2 and its continuation to
    z^4/24 (the related Runge-Kutta methods, Section 3.2). MPE (2) and MPEA (3): the
    largest root modulus of the characteristic polynomial of the related
    Adams-Bashforth method, AB2 and AB3 (Section 3.2 relates MPE and MPEA to AB2 and
    AB3 and finds their stability limits almost equal): rho(zeta) - z sigma(zeta) with
    rho = zeta^2 - zeta, sigma = (3 zeta - 1)/2 (AB2) and rho = zeta^3 - zeta^2,
    sigma = (23 zeta^2 - 16 zeta + 5)/12 (AB3). A reading: the paper plots the
    stability limits but prints no rule, and the library takes the related method's.
    """
    if stepper == HEUNP:
        return lambda z: abs(1.0 + z + 0.5 * z * z)
    if stepper == RK4P:
        return lambda z: abs(1.0 + z * (1.0 + z * (0.5 + z * (1.0 / 6.0 + z / 24.0))))
    if stepper == MICRO_MPE:
        return lambda z: max(abs(r) for r in np.roots([1.0, -1.0 - 1.5 * z, 0.5 * z]))
    if stepper == MICRO_MPEA:
        return lambda z: max(abs(r) for r in np.roots([1.0, -1.0 - 23.0 / 12.0 * z, 16.0 / 12.0 * z,
                                                       -5.0 / 12.0 * z]))
    raise ValueError("micro_stepper must be 0 (HeunP), 1 (RK4P), 2 (MPE) or 3 (MPEA)")


def stability_limit(alpha: float, stepper: int = 0) -> float:
    """Largest s > 0 with growth <= 1 for z = s(-alpha + i) (``_growth``).

    The linearised LL Jacobian has eigenvalues (+-i - alpha) omega (Section 3.2).
    Scans outward from s = 0 and bisects the first exit from the unit disc.
    """
    w = complex(-alpha, 1.0)
    g = _growth(stepper)

    def amp(s):
        return g(s * w)

    s, ds = 0.0, 1e-3
    while amp(s + ds) <= 1.0:
        s += ds
        if s > 10.0:
            raise ValueError("no finite stability limit")
    lo, hi = s, s + ds
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        if amp(mid) <= 1.0:
            lo = mid
        else:
            hi = mid
    return lo


def heun_stability_limit(alpha: float) -> float:
    """Largest s > 0 with |1 + z + z^2/2| <= 1 for z = s(-alpha + i) (HeunP)."""
    return stability_limit(alpha, 0)


def stencil_symbol_max(order: int) -> float:
    """max over theta of the squared symbol of the staggered D_s D_s (times dx^2).

    Order 2: 4 sin^2(theta/2) -> 4. Order 4: ((27 sin(theta/2) - sin(3 theta/2))/12)^2 -> (28/12)^2.
    """
    return 4.0 if order == 2 else (28.0 / 12.0) ** 2


def coef_upper_bound(cfg) -> float:
    return cfg.c0 + sum(abs(t.amp) for t in cfg.terms)


def micro_dt(cfg, dx: float, a_max: Optional[float] = None) -> float:
    """Micro time step dt = safety * s_max(alpha_micro) / omega_max (a reading: the
    paper states only dt <= C_stab dx^2, eq. Cstab), s_max the stability limit of the
    micro stepper (``stability_limit``).

    omega_max = a_max * d * lambda_s / dx^2 bounds the spectral radius of
    -div(a grad) for the staggered stencil; a_max = c0 + sum |amp|.
    """
    lam = stencil_symbol_max(cfg.stencil_order)
    if a_max is None:
        a_max = coef_upper_bound(cfg)
    omega = a_max * cfg.dim * lam / (dx * dx)
    return cfg.dt_safety * stability_limit(cfg.alpha_micro, getattr(cfg, "micro_stepper", 0)) / omega


MACRO_DT_CONSTANT = 0.06


def macro_dt(cfg) -> float:
    """Macro time step: cfg.dt_macro, or 0.06 * DX^2 / (d * a_max) (a reading: the paper
    prints no macro step for these problems)."""
    if cfg.dt_macro > 0:
        return cfg.dt_macro
    DX = min(cfg.L / n for n in list(cfg.n_macro)[: cfg.dim])
    a_max = coef_upper_bound(cfg)
    if getattr(cfg, "coef_fn", None) is not None:
        a_max = 0.0
        for p in range(cfg.n_points):
            geo = box_geometry(cfg, p)
            a_max = max(a_max, float(max(f.max() for f in face_coefficients(cfg, geo))))
    return MACRO_DT_CONSTANT * DX * DX / (cfg.dim * a_max)


# --------------------------------------------------------------------------
# Box geometry
# --------------------------------------------------------------------------


def box_geometry(cfg, p: int) -> Dict:
    """Parameters of the micro problem at macro point p (C-order linear index)."""
    d = cfg.dim
    n = [int(v) for v in list(cfg.n_macro)[:d]]
    idx = np.unravel_index(int(p), n)
    DX = [cfg.L / nk for nk in n]
    eps = float(cfg.eps_field[p]) if cfg.eps_field is not None else float(cfg.eps)
    N = int(cfg.box_n_field[p]) if cfg.box_n_field is not None else int(cfg.box_n)
    dx = eps / cfg.pts_per_eps
    mup = (N - 1) * dx / 2.0
    mu = cfg.mu_over_eps * eps if cfg.mu_over_eps > 0 else 0.8 * mup
    r = 1 if cfg.stencil_order == 2 else 3
    geo = dict(p=int(p), idx=tuple(int(i) for i in idx), DX=DX,
               xc=[idx[k] * DX[k] for k in range(d)], eps=eps, N=N, dx=dx,
               mu_prime=mup, mu=mu, r=r, M=int(cfg.micro_steps))
    # a_max: the bound c0 + sum |amp| of the separable terms, or, for a coefficient
    # function, the maximum over this box's faces
    a_max = None
    if getattr(cfg, "coef_fn", None) is not None:
        a_max = float(max(f.max() for f in face_coefficients(cfg, geo)))
    geo["dt"] = micro_dt(cfg, dx, a_max)
    return geo


def node_offsets(N: int, dx: float, dtype=np.float64) -> np.ndarray:
    """Micro node coordinates xi_j = (j - (N-1)/2) dx, j = 0..N-1 (the box centred on
    its macro point)."""
    return (np.arange(N, dtype=dtype) - dtype(N - 1) / 2) * dtype(dx)


# --------------------------------------------------------------------------
# Micro initial data (Section 4.1, eq. Q_k)
# --------------------------------------------------------------------------


def lagrange_basis(s: np.ndarray, k: int) -> np.ndarray:
    """Lagrange basis l_a(s), a = -k..k, on the integer nodes -k..k; shape (len(s), 2k+1)."""
    s = np.asarray(s)
    if s.dtype.kind != "f":
        s = s.astype(np.float64)
    nodes = np.arange(-k, k + 1)
    out = np.ones((s.size, nodes.size), dtype=s.dtype)
    for ia, a in enumerate(nodes):
        for b in nodes:
            if b != a:
                out[:, ia] *= (s - b) / (a - b)
    return out


def gather_neighbourhood(cfg, M: np.ndarray, idx: Sequence[int]) -> np.ndarray:
    """Macro values M_{i+a}, a in {-k..k}^d with periodic wrap; (3, 2k+1, ...)."""
    d = cfg.dim
    k = cfg.interp_order // 2
    n = [int(v) for v in list(cfg.n_macro)[:d]]
    Mg = M.reshape((3,) + tuple(n))
    ix = [(idx[a] + np.arange(-k, k + 1)) % n[a] for a in range(d)]
    return Mg[np.ix_(range(3), *ix)]


def interpolate_P(neigh: np.ndarray, s_axes: Sequence[np.ndarray], k: int) -> np.ndarray:
    """P_[2k] at the micro nodes, one dimension after the other (Section 4.1).

    neigh: (3, 2k+1, ..., 2k+1); s_axes[a]: node coordinates along axis a in
    units of DX relative to x_i. Returns (3, N_1, ..., N_d).
    """
    P = neigh
    for a, s in enumerate(s_axes):
        L = lagrange_basis(s, k)                      # (N_a, 2k+1)
        P = np.moveaxis(np.tensordot(L, np.moveaxis(P, a + 1, 0), axes=(1, 0)), 0, a + 1)
    return P


def micro_initial(cfg, M: np.ndarray, geo: Dict, normalise: bool = True, dtype=np.float64) -> np.ndarray:
    """m_init = Q_[2k](x_i + xi) = P/|P| on all micro nodes (eq. Q_k)."""
    k = cfg.interp_order // 2
    neigh = gather_neighbourhood(cfg, M, geo["idx"]).astype(dtype)
    xi = node_offsets(geo["N"], geo["dx"], dtype)
    s_axes = [xi / dtype(geo["DX"][a]) for a in range(cfg.dim)]
    P = interpolate_P(neigh, s_axes, k)
    if not normalise:
        return P
    return P / np.sqrt((P ** 2).sum(0))


# --------------------------------------------------------------------------
# Coefficient a^eps (Section 2.1 (A1); workloads' separable-sum form)
# --------------------------------------------------------------------------


def coef_eval(cfg, eps: float, X: Sequence[np.ndarray], dtype=np.float64) -> np.ndarray:
    """a(x) = c0 + sum_t amp_t prod_k g_tk(2 pi omega_tk s_k + phase_tk), s = x/eps or x;
    or the configuration's own coefficient function (cfg.coef_fn) when it has one."""
    if getattr(cfg, "coef_fn", None) is not None:
        return np.broadcast_to(np.asarray(cfg.coef_fn(list(X), eps), dtype=dtype), np.broadcast(*X).shape)
    out = np.full(np.broadcast(*X).shape, dtype(cfg.c0), dtype=dtype)
    two_pi = 2 * _pi(dtype)
    for t in cfg.terms:
        val = np.full_like(out, dtype(t.amp))
        for k in range(cfg.dim):
            if t.kind[k] == 0:
                continue
            s = X[k] / dtype(eps) if t.scale[k] == 0 else X[k]
            th = two_pi * dtype(t.omega[k]) * s + dtype(t.phase[k])
            val = val * (np.sin(th) if t.kind[k] == 1 else np.cos(th))
        out = out + val
    return out


def face_coefficients(cfg, geo: Dict, dtype=np.float64) -> List[np.ndarray]:
    """a^eps at the faces of each axis: for axis k, shape (N,..,N-1 at axis k,..,N).

    Face j+1/2 along axis k lies at xi_k = (j + 1/2 - (N-1)/2) dx, the other
    coordinates at nodes; the coefficient is taken at the face's exact
    coordinate x_i + xi (fast variable with the box's eps).
    """
    d, N, dx = cfg.dim, geo["N"], geo["dx"]
    xi = node_offsets(N, dx, dtype)
    xf = (np.arange(N - 1, dtype=dtype) + dtype(0.5) - dtype(N - 1) / 2) * dtype(dx)
    out = []
    for k in range(d):
        X = []
        for a in range(d):
            v = xf if a == k else xi
            shp = [1] * d
            shp[a] = v.size
            X.append(dtype(geo["xc"][a]) + v.reshape(shp))
        out.append(coef_eval(cfg, geo["eps"], X, dtype))
    return out


# --------------------------------------------------------------------------
# H = div(a grad m): conservative staggered stencil
# --------------------------------------------------------------------------


def _take(arr: np.ndarray, axis: int, start: int, stop: int) -> np.ndarray:
    sl = [slice(None)] * arr.ndim
    sl[axis] = slice(start, stop)
    return arr[tuple(sl)]


def face_gradient(m: np.ndarray, axis: int, dx: float, order: int) -> np.ndarray:
    """D_s m at faces along ``axis`` (array axis of m).

    Order 2: (m_{j+1} - m_j)/dx at faces j+1/2, j = 0..N-2.
    Order 4: (m_{j-1} - 27 m_j + 27 m_{j+1} - m_{j+2})/(24 dx) at faces j+1/2, j = 1..N-3.
    """
    N = m.shape[axis]
    if order == 2:
        return (_take(m, axis, 1, N) - _take(m, axis, 0, N - 1)) / dx
    return (_take(m, axis, 0, N - 3) - 27.0 * _take(m, axis, 1, N - 2)
            + 27.0 * _take(m, axis, 2, N - 1) - _take(m, axis, 3, N)) / (24.0 * dx)


def node_divergence(F: np.ndarray, axis: int, dx: float, order: int) -> np.ndarray:
    """D_s of face fluxes back to the interior nodes along ``axis``."""
    nf = F.shape[axis]
    if order == 2:
        return (_take(F, axis, 1, nf) - _take(F, axis, 0, nf - 1)) / dx
    return (_take(F, axis, 0, nf - 3) - 27.0 * _take(F, axis, 1, nf - 2)
            + 27.0 * _take(F, axis, 2, nf - 1) - _take(F, axis, 3, nf)) / (24.0 * dx)


def field_H(m: np.ndarray, afaces: List[np.ndarray], dx: float, order: int) -> np.ndarray:
    """H = sum_k D_s(a_f D_s m) at the interior nodes; m is (..., 3, N, ..., N).

    Returns (..., 3, N-2r, ..., N-2r). afaces[k] holds a at all faces j+1/2,
    j = 0..N-2, of axis k (broadcast against m's leading axes).
    """
    d = len(afaces)
    r = 1 if order == 2 else 3
    lead = m.ndim - d
    H = 0.0
    for k in range(d):
        ax = lead + k
        G = face_gradient(m, ax, dx, order)
        a = afaces[k]
        if a.ndim == m.ndim - 1:                      # insert the component axis
            a = np.expand_dims(a, lead - 1)
        N = m.shape[ax]
        a_used = _take(a, ax, 0, N - 1) if order == 2 else _take(a, ax, 1, N - 2)
        Hk = node_divergence(a_used * G, ax, dx, order)
        for other in range(d):
            if other != k:
                Hk = _take(Hk, lead + other, r, N - r)
        H = H + Hk
    return H


def exchange_energy(m: np.ndarray, afaces: List[np.ndarray], dx: float, order: int) -> np.ndarray:
    """E_h = 1/2 dx^d sum over the faces used by H of a_f |D_s m|^2.

    These are the faces on lines through interior nodes; for interior nodes
    H = -(1/dx^d) dE_h/dm, so the semi-discrete dE_h/dt = -alpha dx^d sum |m x H|^2.
    """
    d = len(afaces)
    r = 1 if order == 2 else 3
    lead = m.ndim - d
    E = 0.0
    for k in range(d):
        ax = lead + k
        N = m.shape[ax]
        G = face_gradient(m, ax, dx, order)
        a = afaces[k]
        a_used = _take(a, a.ndim - d + k, 0, N - 1) if order == 2 else _take(a, a.ndim - d + k, 1, N - 2)
        e = a_used * (G ** 2).sum(axis=lead - 1)
        for other in range(d):
            if other != k:
                e = _take(e, e.ndim - d + other, r, N - r)
        E = E + e.reshape(e.shape[: e.ndim - d] + (-1,)).sum(-1)
    return 0.5 * dx ** d * E


# --------------------------------------------------------------------------
# Landau-Lifshitz right-hand side and HeunP (Section 3.1)
# --------------------------------------------------------------------------


def ll_rhs(m: np.ndarray, H: np.ndarray, alpha: float, axis: int = 0) -> np.ndarray:
    """f = -m x H - alpha m x (m x H) along the component ``axis``."""
    mxH = np.cross(m, H, axis=axis)
    return -mxH - alpha * np.cross(m, mxH, axis=axis)


def _interior(arr: np.ndarray, d: int, r: int) -> Tuple:
    return (Ellipsis,) + tuple(slice(r, arr.shape[-d + k] - r) for k in range(d))


def midpoint_solve(m: np.ndarray, h: np.ndarray, dt: float, axis: int) -> np.ndarray:
    """m' with (m' - m)/dt = -(m + m')/2 x h at every node (eq. mpe_update).

    As in ``midpoint_update``: with w = dt/2 h and [w]_x v = w x v, (I - [w]_x) m' =
    (I + [w]_x) m, one 3x3 system per node (components along ``axis``), solved by
    Cramer's rule (plain arithmetic, so any working precision).
    """
    mm = np.moveaxis(m, axis, -1)
    w = 0.5 * dt * np.moveaxis(h, axis, -1)
    z = np.zeros_like(w[..., 0])
    one = z + 1
    wx = [[z, -w[..., 2], w[..., 1]],
          [w[..., 2], z, -w[..., 0]],
          [-w[..., 1], w[..., 0], z]]                       # wx @ v = w x v
    A = [[(one if i == j else z) - wx[i][j] for j in range(3)] for i in range(3)]
    b = [mm[..., i] + sum(wx[i][j] * mm[..., j] for j in range(3)) for i in range(3)]

    def det(c0, c1, c2):   # determinant of the matrix with columns c0, c1, c2
        return (c0[0] * (c1[1] * c2[2] - c1[2] * c2[1]) - c1[0] * (c0[1] * c2[2] - c0[2] * c2[1])
                + c2[0] * (c0[1] * c1[2] - c0[2] * c1[1]))

    cols = [[A[i][j] for i in range(3)] for j in range(3)]
    dA = det(*cols)
    out = [det(*[b if j == k else cols[j] for j in range(3)]) / dA for k in range(3)]
    return np.moveaxis(np.stack(out, -1), -1, axis)


def micro_solve(m_init: np.ndarray, afaces: List[np.ndarray], dx: float, dt: float,
                M: int, alpha_micro: float, W: np.ndarray, w: np.ndarray, order: int,
                trace: bool = False, stepper: int = 0, flux: Optional[Tuple[int, np.ndarray]] = None):
    """One batch of micro problems with a common grid; returns H_avg (B, 3).

    m_init: (B, 3, N, ..., N). The micro problem (eq. micro) is stepped by HeunP
    (Section 3.1): k1 = f(m^n), k2 = f(m^n + dt k1) (a reading: the standard
    Heun second stage, the one for which the stated update is second order),
    m~ = m^n + dt/2 (k1 + k2), m^{n+1} = m~/|m~|; with stepper = 1 by RK4P
    (Section 3.1): k1 = f(m^n), k2 = f(m^n + dt/2 k1), k3 = f(m^n + dt/2 k2),
    k4 = f(m^n + dt k3), m~ = m^n + dt/6 (k1 + 2 k2 + 2 k3 + k4), m^{n+1} =
    m~/|m~| (the third stage read as above, where the printed stage repeats
    k_2); with stepper = 2 (MPE) or 3 (MPEA) by the midpoint update with an
    extrapolated h (Section 3.1, eqs. h_term, h_mpe, h_mpea, mpe_update), node by
    node: h^n = H(m^n) + alpha m^n x H(m^n), h^{n+1/2} by ``extrapolate_h`` and
    m^{n+1} from (m^{n+1} - m^n)/dt = -(m^n + m^{n+1})/2 x h^{n+1/2}, after
    start-up steps by RK4P (one for MPE, two for MPEA; a reading: the paper allows
    HeunP or RK4P, and RK4P is what the macro stepper uses). Only interior nodes move;
    ring nodes keep m_init (Dirichlet on m - m_init, Section 4.2).
    The average (eq. upscaling) is sum_n w_n sum_xi W(xi) H(m^n)(xi), with
    H(m^n) the stage-1 field of step n (a reading: the paper does not say which
    stage's field enters); w_0 = w_M = 0.
    W is the (N-2r)^d tensor of interior spatial weights.

    With ``flux = (k, Wf)`` the averaged quantity is instead the flux a^eps D_s m
    along axis k at that axis's faces (the flux model, Section 2.2): Wf is the
    weight tensor over the faces face_gradient returns along k and all nodes
    along the other axes.
    """
    d = len(afaces)
    r = 1 if order == 2 else 3
    cax = m_init.ndim - d - 1
    m = m_init.copy()
    inner = _interior(m, d, r)
    S = np.zeros(m.shape[:cax] + (3,), dtype=m.dtype)
    Wb = W[(None,) * (cax + 1)] if W is not None else None
    red = tuple(range(cax + 1, m.ndim))
    energies, normdev = [], []
    hist: List[np.ndarray] = []   # [h^{n-1}, h^{n-2}] (MPE, MPEA)
    if flux is not None:
        fk, Wf = flux
        fax = cax + 1 + fk
        Nk = m.shape[fax]
        af = afaces[fk]
        if af.ndim == m.ndim - 1:
            af = np.expand_dims(af, cax)
        af = _take(af, fax, 0, Nk - 1) if order == 2 else _take(af, fax, 1, Nk - 2)
        Wfb = Wf[(None,) * (cax + 1)]
    for n in range(M + 1):
        H1 = field_H(m, afaces, dx, order)
        if w[n] != 0.0:
            if flux is None:
                S += w[n] * (Wb * H1).sum(axis=red)
            else:
                S += w[n] * (Wfb * (af * face_gradient(m, fax, dx, order))).sum(axis=red)
        if trace:
            energies.append(exchange_energy(m, afaces, dx, order))
            normdev.append(np.abs(np.sqrt((m ** 2).sum(cax)) - 1.0).max())
        if n == M:
            break
        mi = m[inner]
        k1 = ll_rhs(mi, H1, alpha_micro, axis=cax)

        def stage(c, k):
            # f at the stage state m + c k (ring nodes keep m_init)
            ms = m.copy()
            ms[inner] = mi + c * k
            return ll_rhs(ms[inner], field_H(ms, afaces, dx, order), alpha_micro, axis=cax)

        if stepper >= MICRO_MPE:
            hn = H1 + alpha_micro * np.cross(mi, H1, axis=cax)   # eq. h_term at m^n
            if n >= (1 if stepper == MICRO_MPE else 2):
                hx = extrapolate_h(hn, hist, MPE if stepper == MICRO_MPE else MPEA)
                m[inner] = midpoint_solve(mi, hx, dt, cax)
                hist = [hn] + hist[:1]
                continue
            hist = [hn] + hist[:1]
        if stepper == 0:
            k2 = stage(dt, k1)
            mt = mi + 0.5 * dt * (k1 + k2)
        else:
            k2 = stage(0.5 * dt, k1)
            k3 = stage(0.5 * dt, k2)
            k4 = stage(dt, k3)
            mt = mi + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        m[inner] = mt / np.sqrt((mt ** 2).sum(cax, keepdims=True))
    if trace:
        return S, m, np.array(energies), np.array(normdev)
    return S


# --------------------------------------------------------------------------
# The batched micro solve: one H_avg per macro point (eq. upscaling)
# --------------------------------------------------------------------------


def micro_batch(cfg, M: np.ndarray, points: Optional[Sequence[int]] = None,
                group: int = 64, dtype=np.float64) -> np.ndarray:
    """H_avg(x_i; M) for macro points ``points`` (default all); returns (3, len).

    ``dtype`` is the working precision (FP64 by default; np.longdouble gives a
    reference with a lower rounding floor, used to bound the FP64 results' own
    rounding error).
    """
    P = cfg.n_points
    pts = list(range(P)) if points is None else [int(p) for p in points]
    out = np.zeros((3, len(pts)), dtype=dtype)
    geos = [box_geometry(cfg, p) for p in pts]
    keys: Dict[Tuple, List[int]] = {}
    for i, g in enumerate(geos):
        keys.setdefault((g["N"], g["dx"], g["dt"], g["mu"]), []).append(i)
    for (N, dx, dt, mu), members in keys.items():
        d, r = cfg.dim, geos[members[0]]["r"]
        Wfull = space_weights(N, dx, mu, cfg.px, cfg.qx, dtype)
        if np.any(Wfull[:r] != 0.0) or np.any(Wfull[N - r:] != 0.0):
            raise ValueError("averaging box [-mu, mu] reaches the Dirichlet ring")
        W1 = Wfull[r:N - r]
        W = W1
        for _ in range(d - 1):
            W = np.multiply.outer(W, W1)
        w = time_weights(cfg.micro_steps, cfg.pt, cfg.qt, dtype)
        for s in range(0, len(members), group):
            chunk = members[s:s + group]
            mi = np.stack([micro_initial(cfg, M, geos[i], dtype=dtype) for i in chunk])
            af = [np.stack([face_coefficients(cfg, geos[i], dtype)[k] for i in chunk]) for k in range(d)]
            S = micro_solve(mi, af, dtype(dx), dtype(dt), cfg.micro_steps, dtype(cfg.alpha_micro),
                            W, w, cfg.stencil_order, stepper=getattr(cfg, "micro_stepper", 0))
            for j, i in enumerate(chunk):
                out[:, i] = S[j]
    return out


# --------------------------------------------------------------------------
# Macro time stepping (Section 3.1: HeunP/RK4P, MPEA; Section 3.3)
# --------------------------------------------------------------------------


def _normalise(M: np.ndarray) -> np.ndarray:
    return M / np.sqrt((M ** 2).sum(0, keepdims=True))


def h_term(M: np.ndarray, H: np.ndarray, alpha: float) -> np.ndarray:
    """h = H + alpha M x H (eq. h_term)."""
    return H + alpha * np.cross(M, H, axis=0)


def midpoint_update(M: np.ndarray, h: np.ndarray, dt: float) -> np.ndarray:
    """Solve (M' - M)/dt = -(M + M')/2 x h for M' per point (eq. mpe_update).

    Rearranged: M' + (dt/2) M' x h = M - (dt/2) M x h, a 3x3 linear system per
    point, solved directly (a reading: the signs of eq. mpe_update and
    eq. imp_update, not of eq. imp_sys).
    """
    P = M.shape[1]
    w = 0.5 * dt * h
    out = np.empty_like(M)
    for p in range(P):
        wx = np.array([[0.0, -w[2, p], w[1, p]],
                       [w[2, p], 0.0, -w[0, p]],
                       [-w[1, p], w[0, p], 0.0]])       # wx @ v = w x v
        # M' x h (dt/2) = -(w x M'); so (I - wx) M' = (I + wx) M
        A = np.eye(3) - wx
        b = (np.eye(3) + wx) @ M[:, p]
        out[:, p] = np.linalg.solve(A, b)
    return out


MPEA, MPE = 0, 1   # macro steppers (Section 3.1)


def extrapolate_h(hj: np.ndarray, hist: Sequence[np.ndarray], scheme: int = MPEA) -> np.ndarray:
    """The explicit stand-in h^{j+1/2} for h at the midpoint of step j (Section 3.1).

    MPE (eq. h_mpe): 3/2 h^j - 1/2 h^{j-1}. MPEA (eq. h_mpea): 23/12 h^j -
    16/12 h^{j-1} + 5/12 h^{j-2}. ``hist`` = [h^{j-1}, h^{j-2}] (h^{j-2} unused by MPE).
    The coefficients are those of Adams-Bashforth 2 and 3, the methods the paper
    links MPE and MPEA to (Section 3.2, eq. mpe_update_ab).
    """
    if scheme == MPE:
        return 1.5 * hj - 0.5 * hist[0]
    return 23.0 / 12.0 * hj - 16.0 / 12.0 * hist[0] + 5.0 / 12.0 * hist[1]


class MacroStepper:
    """Field-model HMM macro stepper (eq. macro_disc): MPEA or MPE with RK4P start-up.

    ``havg(M)`` returns H_avg(x_i; M) for all macro points (default: the
    oracle's micro_batch). The first steps use RK4P (Section 3.1; the third stage
    read as f(M + dt/2 k2) where the printed stage repeats k_2) whose stage states
    are normalised before their micro solves (a reading: assumption A3 for the
    micro initial data): j = 0, 1 for MPEA, which needs h^{j-1} and h^{j-2}, and
    j = 0 for MPE, which needs h^{j-1} only (Section 3.1: the multi-step methods
    need m^1, and m^2 for MPEA). Then h^j = H_avg + alpha M x H_avg (eq. h_term),
    h^{j+1/2} by ``extrapolate_h`` and the midpoint update (eq. mpe_update).
    ``scheme``: MPEA (0) or MPE (1); default the config's ``macro_stepper``.
    """

    def __init__(self, cfg, M0: np.ndarray, havg=None, dt: Optional[float] = None,
                 scheme: Optional[int] = None):
        self.cfg = cfg
        self.M = np.array(M0, dtype=np.float64, copy=True)
        self.havg = havg if havg is not None else (lambda M: micro_batch(cfg, M))
        self.dt = macro_dt(cfg) if dt is None else dt
        self.scheme = int(getattr(cfg, "macro_stepper", MPEA) if scheme is None else scheme)
        self.n_startup = 1 if self.scheme == MPE else 2
        self.j = 0
        self.hist: List[np.ndarray] = []   # [h^{j-1}, h^{j-2}]

    def _f(self, M, H):
        return ll_rhs(M, H, self.cfg.alpha, axis=0)

    def step(self):
        a, dt, M = self.cfg.alpha, self.dt, self.M
        if self.j < self.n_startup:
            H1 = self.havg(M)
            hj = h_term(M, H1, a)
            k1 = self._f(M, H1)
            M2 = _normalise(M + 0.5 * dt * k1)
            k2 = self._f(M2, self.havg(M2))
            M3 = _normalise(M + 0.5 * dt * k2)
            k3 = self._f(M3, self.havg(M3))
            M4 = _normalise(M + dt * k3)
            k4 = self._f(M4, self.havg(M4))
            self.M = _normalise(M + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4))
        else:
            hj = h_term(M, self.havg(M), a)
            self.M = midpoint_update(M, extrapolate_h(hj, self.hist, self.scheme), dt)
        self.hist = [hj] + self.hist[:1]
        self.j += 1
        return self.M


# --------------------------------------------------------------------------
# Homogenised targets (Section 2.1 eqs. AH, cell_problem; Theorem 2)
# --------------------------------------------------------------------------


def q_derivatives_at_centre(cfg, M: np.ndarray, p: int, return_p: bool = False):
    """First and second derivatives of Q_[2k](x_i + xi) at xi = 0, (3, d) and (3, d, d).

    Uses the exact derivatives of the Lagrange polynomials (P', P'') and the
    quotient rule for Q = P/|P| (Section 4.1, proof of the Lemma). With
    ``return_p`` the un-normalised P, P', P'' are returned instead.
    """
    d, k = cfg.dim, cfg.interp_order // 2
    geo = box_geometry(cfg, p)
    neigh = gather_neighbourhood(cfg, M, geo["idx"])
    nodes = np.arange(-k, k + 1)
    # values, first and second derivative of the 1D basis at s = 0 (units of DX)
    L0 = lagrange_basis(np.array([0.0]), k)[0]
    coef = [np.polynomial.polynomial.polyfromroots([b for b in nodes if b != a]) /
            np.prod([a - b for b in nodes if b != a]) for a in nodes]
    L1 = np.array([np.polynomial.polynomial.polyval(0.0, np.polynomial.polynomial.polyder(c, 1)) for c in coef])
    L2 = np.array([np.polynomial.polynomial.polyval(0.0, np.polynomial.polynomial.polyder(c, 2)) for c in coef])
    DX = geo["DX"]

    def apply(orders):
        # contract the spatial axes one after the other with the basis derivative
        T = neigh
        for a in range(d):
            vec = [L0, L1, L2][orders[a]] / DX[a] ** orders[a]
            T = np.tensordot(T, vec, axes=([1], [0]))
        return T

    Pv = apply([0] * d)
    P1 = np.stack([apply([1 if a == b else 0 for a in range(d)]) for b in range(d)], -1)
    P2 = np.zeros((3, d, d))
    for a in range(d):
        for b in range(d):
            o = [0] * d
            o[a] += 1
            o[b] += 1
            P2[:, a, b] = apply(o)
    if return_p:
        return Pv, P1, P2
    n = np.linalg.norm(Pv)
    # Q = P/|P|: d_a Q = P_a/n - (P.P_a) P/n^3
    Q1 = P1 / n - np.outer(Pv, Pv @ P1) / n ** 3
    Q2 = np.zeros((3, d, d))
    for a in range(d):
        for b in range(d):
            pa, pb, pab = P1[:, a], P1[:, b], P2[:, a, b]
            Q2[:, a, b] = (pab / n - (Pv @ pb) * pa / n ** 3 - (Pv @ pa) * pb / n ** 3
                           - ((pa @ pb) + (Pv @ pab)) * Pv / n ** 3
                           + 3.0 * (Pv @ pa) * (Pv @ pb) * Pv / n ** 5)
    return Pv / n, Q1, Q2


def homogenised_target(AH: np.ndarray, Q2: np.ndarray) -> np.ndarray:
    """div(grad m_init(0) A^H) = sum_kl A^H_kl d_k d_l m_init(0) (Theorem 2)."""
    return np.einsum("kl,ckl->c", AH, Q2)
