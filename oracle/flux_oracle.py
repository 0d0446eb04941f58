"""Plain FP64 CPU oracle of the HMM flux model.

TEST INFRASTRUCTURE ONLY, like ``hmm_oracle``: imported by ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline/reference leg, and
by nothing else. The CUDA library never imports, links or executes it.

The flux model (Section 2.2, eq. macro_flux) evolves the macro state by
dM/dt = -M x div F_avg - alpha M x (M x div F_avg), where F_avg approximates
grad m A^H: the same kernel-weighted space-time average (eq. upscaling) as the
field model's, applied to the flux a^eps grad m of the micro solution instead
of to div(a^eps grad m). The paper places the flux components at different
grid locations so that the macro divergence is a compact difference, which
takes one micro problem per gradient component. This module computes, step by
step, with the micro problem, kernels, weights and time stepping of
``hmm_oracle``:

* column k of F_avg at the staggered point x_i + (DX_k/2) e_k, from a micro
  problem centred there (reading: initial data = the interpolant Q_[2k] of the
  macro neighbourhood of x_i, evaluated at the shifted nodes; the coefficient
  at the true positions; the micro time step of the field model);
* the average of the face flux a_f D_s m along axis k over that axis's faces,
  with the spatial kernel evaluated at the face positions (trapezoid weights,
  normalised to sum 1 like the node weights: the paper fixes no quadrature);
* the macro divergence (div F)_i = sum_k D_k F_k by the staggered difference of
  the same order as the interpolation (reading: order 4 for Q_[4], order 2 for
  Q_[2]), periodic;
* the macro step: ``hmm_oracle.MacroStepper`` with div F_avg in place of H_avg.
"""
from __future__ import annotations

from typing import Dict, Optional, Sequence

import numpy as np

from . import hmm_oracle as O


def flux_geometry(cfg, p: int, k: int) -> Dict:
    """The micro problem for column k of F_avg at the staggered point of macro
    point p: box_geometry's, centred at x_p + (DX_k/2) e_k."""
    geo = dict(O.box_geometry(cfg, p))
    geo["xc"] = list(geo["xc"])
    geo["xc"][k] += geo["DX"][k] / 2.0
    geo["shift"] = [0.5 if a == k else 0.0 for a in range(cfg.dim)]
    geo["axis"] = k
    if getattr(cfg, "coef_fn", None) is not None:
        a_max = float(max(f.max() for f in O.face_coefficients(cfg, geo)))
        geo["dt"] = O.micro_dt(cfg, geo["dx"], a_max)
    return geo


def flux_initial(cfg, M: np.ndarray, geo: Dict, dtype=np.float64) -> np.ndarray:
    """m_init = Q_[2k] at the shifted micro nodes: the interpolant of the
    neighbourhood of x_p at s = xi/DX + shift (Section 4.1, eq. Q_k)."""
    k = cfg.interp_order // 2
    neigh = O.gather_neighbourhood(cfg, M, geo["idx"]).astype(dtype)
    xi = O.node_offsets(geo["N"], geo["dx"], dtype)
    s_axes = [xi / dtype(geo["DX"][a]) + dtype(geo["shift"][a]) for a in range(cfg.dim)]
    P = O.interpolate_P(neigh, s_axes, k)
    return P / np.sqrt((P ** 2).sum(0))


def face_weights(N: int, dx: float, mu: float, p: int, q: int, dtype=np.float64) -> np.ndarray:
    """Weights of K_mu at the faces xi_j + dx/2, j = 0..N-2 (trapezoid rule,
    normalised to sum 1)."""
    xf = (np.arange(N - 1, dtype=dtype) + dtype(0.5) - dtype(N - 1) / 2) * dtype(dx)
    W = O.kernel_eval(xf / dtype(mu), p, q, dtype)
    return W / W.sum()


def micro_batch_flux(cfg, M: np.ndarray, points: Optional[Sequence[int]] = None,
                     axes: Optional[Sequence[int]] = None, dtype=np.float64) -> np.ndarray:
    """Columns k of F_avg at the staggered points of macro points ``points``;
    returns (len(axes), 3, len(points))."""
    d = cfg.dim
    P = cfg.n_points
    pts = list(range(P)) if points is None else [int(p) for p in points]
    axes = list(range(d)) if axes is None else list(axes)
    out = np.zeros((len(axes), 3, len(pts)), dtype=dtype)
    w = O.time_weights(cfg.micro_steps, cfg.pt, cfg.qt, dtype)
    for ia, k in enumerate(axes):
        for ip, p in enumerate(pts):
            geo = flux_geometry(cfg, p, k)
            N, dx, r = geo["N"], geo["dx"], geo["r"]
            Wn = O.space_weights(N, dx, geo["mu"], cfg.px, cfg.qx, dtype)
            Wf = face_weights(N, dx, geo["mu"], cfg.px, cfg.qx, dtype)
            if np.any(Wn[:r] != 0.0) or np.any(Wn[N - r:] != 0.0):
                raise ValueError("averaging box [-mu, mu] reaches the Dirichlet ring")
            # faces with weight: those touching an interior node, j = r-1..N-r-1 (implied by
            # the node condition above: the next face out lies beyond a ring node)
            if np.any(Wf[:r - 1] != 0.0) or np.any(Wf[N - r:] != 0.0):
                raise ValueError("averaging box [-mu, mu] reaches a face between ring nodes")
            Wk = Wf[0:N - 1] if cfg.stencil_order == 2 else Wf[1:N - 2]   # faces face_gradient returns
            Wt = None
            for a in range(d):
                v = Wk if a == k else Wn
                Wt = v if Wt is None else np.multiply.outer(Wt, v)
            mi = flux_initial(cfg, M, geo, dtype)[None]
            af = [f[None] for f in O.face_coefficients(cfg, geo, dtype)]
            S = O.micro_solve(mi, af, dtype(dx), dtype(geo["dt"]), cfg.micro_steps, dtype(cfg.alpha_micro),
                              None, w, cfg.stencil_order, stepper=getattr(cfg, "micro_stepper", 0),
                              flux=(k, Wt))
            out[ia, :, ip] = S[0]
    return out


def flux_divergence(cfg, F: np.ndarray) -> np.ndarray:
    """(div F)_i = sum_k D_k F_k on the periodic macro grid; F is (d, 3, P) with
    F[k][:, p] the flux column k at x_p + (DX_k/2) e_k. Staggered difference of
    order interp_order: order 4 (F_{i-3/2} - 27 F_{i-1/2} + 27 F_{i+1/2} -
    F_{i+3/2})/(24 DX), order 2 (F_{i+1/2} - F_{i-1/2})/DX. Returns (3, P)."""
    d = cfg.dim
    n = [int(v) for v in list(cfg.n_macro)[:d]]
    out = np.zeros((3,) + tuple(n), dtype=F.dtype)
    for k in range(d):
        Fk = F[k].reshape((3,) + tuple(n))
        ax = 1 + k
        DX = cfg.L / n[k]

        def sh(s):   # F at face i + 1/2 + s (entry i is face i + 1/2)
            return np.roll(Fk, -s, axis=ax)
        if cfg.interp_order == 2:
            out += (Fk - sh(-1)) / DX
        else:
            out += (sh(-2) - 27.0 * sh(-1) + 27.0 * Fk - sh(1)) / (24.0 * DX)
    return out.reshape(3, -1)


def flux_field(cfg, M: np.ndarray, dtype=np.float64) -> np.ndarray:
    """div F_avg(M) at every macro point, the flux model's counterpart of H_avg."""
    return flux_divergence(cfg, micro_batch_flux(cfg, M, dtype=dtype))


def macro_stepper(cfg, M0: np.ndarray, dt: Optional[float] = None) -> O.MacroStepper:
    """The flux model's macro stepper (eq. macro_flux): MPEA with RK4P start-up."""
    return O.MacroStepper(cfg, M0, havg=lambda M: flux_field(cfg, M), dt=dt)
