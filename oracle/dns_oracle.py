"""Plain FP64 CPU oracle of the direct simulation resolving eps.

TEST INFRASTRUCTURE ONLY, like ``hmm_oracle``: imported by ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline/reference leg, and
by nothing else. The CUDA library never imports, links or executes it.

The paper's reference solutions M^eps (Section 5, the locally periodic 1D and
the quasi-periodic 2D examples) come from a direct simulation of eq. prob on
the periodic domain [0, L]^d with a grid that resolves eps (15 points per eps
there), time-stepped by MPEA. This module computes exactly that, step by step:

* the grid x_j = j dx, dx = L/n per axis, periodic in every axis;
* a^eps at the staggered faces x_j + (dx/2) e_k, from the same separable
  coefficient description as the micro problems (or a coefficient function);
* H = div(a^eps grad m) by the conservative staggered difference of the micro
  problems (order 2 as in Section 2.3, or order 4), here with periodic wrap
  instead of the Dirichlet ring;
* the field model's time stepping (Section 3.1): two RK4P start-up steps with
  normalised stage states, then MPEA (eqs. h_term, h_mpea, mpe_update), with
  H in place of H_avg. The stepper is ``hmm_oracle.MacroStepper`` itself.

The default time step is a reading (the paper prints none for its direct
simulations): half the largest step for which the third-order Adams-Bashforth
extrapolation that MPEA uses is stable on the linearised spectrum
omega (-alpha +- i), omega <= d a_max lambda_s / dx^2.
"""
from __future__ import annotations

import types
from typing import List, Optional, Sequence

import numpy as np

from . import hmm_oracle as O

# --------------------------------------------------------------------------
# Grid and coefficient
# --------------------------------------------------------------------------


def grid_spacing(cfg) -> List[float]:
    """dx_k = L / n_k per axis."""
    return [cfg.L / int(n) for n in list(cfg.n)[: cfg.dim]]


def face_coefficients(cfg, index: Optional[Sequence[np.ndarray]] = None,
                      dtype=np.float64) -> List[np.ndarray]:
    """a^eps at the faces x_j + (dx/2) e_k of axis k, one array per axis.

    ``index`` gives the global node indices along each axis (default: the whole
    grid, arange(n_k)); the result for axis k has the shape of the index grid,
    entry j holding a at the face between node j and node j + e_k.
    """
    d = cfg.dim
    dx = grid_spacing(cfg)
    if index is None:
        index = [np.arange(int(n)) for n in list(cfg.n)[:d]]
    out = []
    for k in range(d):
        X = []
        for a in range(d):
            shp = [1] * d
            shp[a] = len(index[a])
            x = np.asarray(index[a], dtype=dtype) * dtype(dx[a])
            if a == k:
                x = x + dtype(0.5) * dtype(dx[a])
            X.append(x.reshape(shp))
        out.append(np.broadcast_to(O.coef_eval(cfg, cfg.eps, X, dtype),
                                   tuple(len(i) for i in index)).copy())
    return out


# --------------------------------------------------------------------------
# Periodic staggered stencil
# --------------------------------------------------------------------------


def _shift(u: np.ndarray, s: int, axis: int) -> np.ndarray:
    """u_{j+s} along ``axis`` with periodic wrap."""
    return np.roll(u, -s, axis=axis)


def face_gradient(m: np.ndarray, axis: int, dx: float, order: int) -> np.ndarray:
    """D_s m at the faces j + 1/2 along ``axis`` (entry j), periodic.

    Order 2: (m_{j+1} - m_j)/dx. Order 4: (m_{j-1} - 27 m_j + 27 m_{j+1} - m_{j+2})/(24 dx).
    """
    if order == 2:
        return (_shift(m, 1, axis) - m) / dx
    return (_shift(m, -1, axis) - 27.0 * m + 27.0 * _shift(m, 1, axis)
            - _shift(m, 2, axis)) / (24.0 * dx)


def node_divergence(F: np.ndarray, axis: int, dx: float, order: int) -> np.ndarray:
    """D_s of face values (entry j = face j + 1/2) back to the nodes, periodic.

    Order 2: (F_{j+1/2} - F_{j-1/2})/dx. Order 4:
    (F_{j-3/2} - 27 F_{j-1/2} + 27 F_{j+1/2} - F_{j+3/2})/(24 dx).
    """
    if order == 2:
        return (F - _shift(F, -1, axis)) / dx
    return (_shift(F, -2, axis) - 27.0 * _shift(F, -1, axis) + 27.0 * F
            - _shift(F, 1, axis)) / (24.0 * dx)


def field_H(m: np.ndarray, afaces: Sequence[np.ndarray], dx: Sequence[float], order: int) -> np.ndarray:
    """H = sum_k D_s(a_f D_s m) along each axis; m is (3, n_1, .., n_d), periodic."""
    H = np.zeros_like(m)
    for k, a in enumerate(afaces):
        ax = 1 + k
        H = H + node_divergence(a[None] * face_gradient(m, ax, dx[k], order), ax, dx[k], order)
    return H


def exchange_energy(m: np.ndarray, afaces: Sequence[np.ndarray], dx: Sequence[float], order: int) -> float:
    """E_h = 1/2 (prod dx) sum over all faces of a_f |D_s m|^2 (periodic)."""
    E = 0.0
    for k, a in enumerate(afaces):
        G = face_gradient(m, 1 + k, dx[k], order)
        E += float((a * (G ** 2).sum(0)).sum())
    return 0.5 * float(np.prod(dx)) * E


# --------------------------------------------------------------------------
# Time step (reading: the paper prints none for the direct simulation)
# --------------------------------------------------------------------------


def ab3_stability_limit(alpha: float) -> float:
    """Largest s > 0 such that the AB3 recurrence
    y_{j+1} = y_j + z (23 y_j - 16 y_{j-1} + 5 y_{j-2})/12, z = s(-alpha + i),
    has all characteristic roots in the closed unit disc (the linearisation of
    MPEA's extrapolated midpoint step). Scan outward from 0, then bisect."""
    w = complex(-alpha, 1.0)

    def rho(s):
        z = s * w
        roots = np.roots([1.0, -1.0 - 23.0 * z / 12.0, 16.0 * z / 12.0, -5.0 * z / 12.0])
        return max(abs(r) for r in roots)

    s, ds = 0.0, 1e-3
    while rho(s + ds) <= 1.0 + 1e-12:
        s += ds
        if s > 10.0:
            raise ValueError("no finite stability limit")
    lo, hi = s, s + ds
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if rho(mid) <= 1.0 + 1e-12:
            lo = mid
        else:
            hi = mid
    return lo


def coef_max(cfg) -> float:
    """Largest face coefficient of the grid (the bound c0 + sum |amp| for separable terms)."""
    if getattr(cfg, "coef_fn", None) is not None:
        return float(max(a.max() for a in face_coefficients(cfg)))
    return O.coef_upper_bound(cfg)


def dns_dt(cfg) -> float:
    """cfg.dt, or safety * s_AB3(alpha) / omega_max with omega_max =
    a_max sum_k lambda_s / dx_k^2 (lambda_s the stencil's largest squared symbol)."""
    if cfg.dt > 0:
        return cfg.dt
    lam = O.stencil_symbol_max(cfg.stencil_order)
    omega = coef_max(cfg) * sum(lam / (h * h) for h in grid_spacing(cfg))
    return cfg.dt_safety * ab3_stability_limit(cfg.alpha) / omega


# --------------------------------------------------------------------------
# The direct simulation
# --------------------------------------------------------------------------


class DNS:
    """M^eps on the periodic grid, advanced by RK4P (steps 0, 1) then MPEA.

    ``M0`` is (3, n_1 .. n_d) or (3, prod n); ``afaces`` overrides the face
    coefficients (default: face_coefficients(cfg)), ``dt`` dns_dt(cfg), and
    ``shape``/``dx`` the grid (used for patches of a larger grid).
    """

    def __init__(self, cfg, M0: np.ndarray, afaces=None, dt: Optional[float] = None,
                 shape: Optional[Sequence[int]] = None, dx: Optional[Sequence[float]] = None):
        self.cfg = cfg
        self.shape = tuple(int(n) for n in (shape if shape is not None else list(cfg.n)[: cfg.dim]))
        self.dx = list(dx) if dx is not None else grid_spacing(cfg)
        self.afaces = face_coefficients(cfg) if afaces is None else afaces
        self.dt = dns_dt(cfg) if dt is None else dt
        shape = (3,) + self.shape

        def field(Mflat):
            return field_H(Mflat.reshape(shape), self.afaces, self.dx, cfg.stencil_order).reshape(3, -1)

        self.stepper = O.MacroStepper(types.SimpleNamespace(alpha=cfg.alpha),
                                      np.asarray(M0, dtype=np.float64).reshape(3, -1), havg=field, dt=self.dt)

    @property
    def M(self) -> np.ndarray:
        return self.stepper.M

    @property
    def j(self) -> int:
        return self.stepper.j

    def step(self, n: int = 1) -> np.ndarray:
        for _ in range(n):
            self.stepper.step()
        return self.stepper.M

    def energy(self) -> float:
        return exchange_energy(self.M.reshape((3,) + self.shape), self.afaces, self.dx,
                               self.cfg.stencil_order)


def patch_run(cfg, M0: np.ndarray, centre: Sequence[int], steps: int, dt: float) -> np.ndarray:
    """M after ``steps`` steps at the grid point ``centre``, computed on a patch.

    A value of H at a node reads nodes at most r = 3 (order 4; 1 for order 2)
    away along each axis, so after the two RK4P steps (4 evaluations each) and
    steps - 2 MPEA steps (one each) the centre depends only on nodes within
    R = r (8 + max(steps - 2, 0)) of it. The oracle runs the same scheme on the
    (2R+2)^d patch of global nodes around the centre (indices taken modulo n,
    face coefficients at their true positions); its own periodic wrap corrupts
    only nodes more than R from the centre. Returns (3,).
    """
    d = cfg.dim
    r = 1 if cfg.stencil_order == 2 else 3
    R = r * (4 * min(steps, 2) + max(steps - 2, 0)) + 1
    shape = tuple(int(n) for n in list(cfg.n)[:d])
    index = [np.arange(centre[a] - R, centre[a] + R + 2) % shape[a] for a in range(d)]
    M0g = np.asarray(M0, dtype=np.float64).reshape((3,) + shape)
    patch = M0g[np.ix_(range(3), *index)]
    pshape = tuple(len(i) for i in index)
    run = DNS(cfg, patch, afaces=face_coefficients(cfg, index), dt=dt, shape=pshape,
              dx=grid_spacing(cfg))
    run.step(steps)
    return run.M.reshape((3,) + pshape)[(slice(None),) + (R,) * d]
