"""Seeded synthetic inputs for the HMM micro-problem path.

This module is shared by the CUDA path's tests/bench and by the oracle. It holds
problem *descriptions* (parameters, coefficient terms) and seeded generators of
macro magnetisation fields. It holds none of the method's arithmetic: no
kernels, weights, interpolation, stencils, time stepping or averaging.

Workloads follow the paper's problem statement (Section 2.1, eq. prob): a
periodic domain [0, L]^d, a coefficient a^eps that oscillates on the scale eps,
damping alpha and unit-length initial data (assumption A3). The named
configurations below carry the shapes, sizes and value distributions of the
paper's examples (Section 2.4 EX1-EX3, Section 5) at the benchmark's
sizes.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence

import numpy as np

__all__ = [
    "CoefTerm", "HMMConfig", "config", "CONFIG_NAMES", "fourier_field",
    "ex1_initial", "ex2_initial", "c1_initial", "uneven_eps_and_n",
    "macro_coords", "DNSConfig", "dns_config", "DNS_NAMES", "dns_initial",
]

# Coefficient factor kinds and variable scales (per axis of a term).
KIND_ONE, KIND_SIN, KIND_COS = 0, 1, 2
SCALE_FAST, SCALE_SLOW = 0, 1


@dataclasses.dataclass
class CoefTerm:
    """One term amp * prod_k g_k(2*pi*omega_k*s_k + phase_k) of a(x).

    g_k is 1, sin or cos (``kind``); s_k = x_k/eps (fast variable, ``scale`` 0)
    or s_k = x_k (slow variable, ``scale`` 1). Axes beyond the problem's
    dimension must have kind 1 (the factor 1).
    """
    amp: float
    kind: Sequence[int] = (KIND_ONE, KIND_ONE, KIND_ONE)
    scale: Sequence[int] = (SCALE_FAST, SCALE_FAST, SCALE_FAST)
    omega: Sequence[float] = (1.0, 1.0, 1.0)
    phase: Sequence[float] = (0.0, 0.0, 0.0)


@dataclasses.dataclass
class HMMConfig:
    """Parameters of one HMM problem (the fields of the C struct hmm_params).

    dim, n_macro, L          periodic macro domain [0, L]^dim, n_macro points/axis
    alpha, alpha_micro       macro damping and artificial micro damping
    dt_macro                 macro time step (<= 0: library/oracle default)
    c0, terms                a(x) = c0 + sum(terms)
    eps / eps_field          uniform eps or one eps per macro point (C order)
    box_n / box_n_field      micro nodes per axis (ring included), uniform or per point
    pts_per_eps              K: micro grid spacing dx = eps/K
    mu_over_eps              averaging half-width mu/eps (<= 0: mu = 0.8*mu')
    micro_steps              M: micro time steps per micro problem (eta = M*dt)
    dt_safety                micro dt as a fraction of the stepper's stability limit
    px, qx, pt, qt           kernel parameters of K in K^{px,qx}, K0 in K0^{pt,qt}
    interp_order             2k of the normalised interpolation Q_[2k]
    stencil_order            2 or 4
    precision                0: plain FP64 method, 1: batched FP32 form
    micro_stepper            0: HeunP, 1: RK4P (Section 3.1) for the micro problems
    model                    0: field model (H_avg), 1: flux model (F_avg at staggered
                             points, its macro divergence in place of H_avg; Section 2.2)
    macro_stepper            0: MPEA, 1: MPE (Section 3.1) for the macro steps
    tile_rows                resident 2D kernel: rows per thread tile (0 tuned, 2 or 4)
    coef_fn                  a coefficient that is not a sum of separable terms:
                             coef_fn(X, eps) -> a at the points X (a list of d
                             coordinate arrays); replaces c0 + terms when set
    """
    dim: int
    n_macro: Sequence[int]
    alpha: float
    alpha_micro: float
    c0: float
    terms: List[CoefTerm]
    eps: float
    box_n: int
    pts_per_eps: float
    micro_steps: int
    L: float = 1.0
    dt_macro: float = 0.0
    eps_field: Optional[np.ndarray] = None
    box_n_field: Optional[np.ndarray] = None
    mu_over_eps: float = 0.0
    dt_safety: float = 0.8
    px: int = 3
    qx: int = 7
    pt: int = 3
    qt: int = 7
    interp_order: int = 4
    stencil_order: int = 4
    precision: int = 0
    micro_stepper: int = 0
    model: int = 0
    macro_stepper: int = 0
    tile_rows: int = 0
    coef_fn: Optional[Callable] = None
    name: str = ""

    @property
    def n_points(self) -> int:
        return int(np.prod(list(self.n_macro)[: self.dim]))

    def replace(self, **kw) -> "HMMConfig":
        return dataclasses.replace(self, **kw)


def macro_coords(cfg: HMMConfig) -> List[np.ndarray]:
    """Macro grid coordinates x_i = i*DX per axis (x_0 = 0)."""
    return [np.arange(n) * (cfg.L / n) for n in list(cfg.n_macro)[: cfg.dim]]


def _grid(cfg: HMMConfig):
    xs = macro_coords(cfg)
    return np.meshgrid(*xs, indexing="ij")


# --------------------------------------------------------------------------
# Seeded initial data
# --------------------------------------------------------------------------

def fourier_field(cfg: HMMConfig, seed: int, kmax: int = 4, sigma: float = 0.5,
                  offset=(0.3, 0.2, 0.9), min_norm: float = 0.25) -> np.ndarray:
    """Normalised smooth random Fourier field on the macro grid, (3, *n_macro).

    m~_c(x) = o_c + sum_{0<|k|<=kmax} sigma/(1+|k|^2) (A cos 2pi k.x + B sin 2pi k.x)
    with A, B ~ N(0,1) drawn from numpy PCG64(seed); redrawn while
    min |m~| < min_norm, with sigma multiplied by 0.7 after every 16 rejected
    draws (2D fields pass within the first 16; 3D fields at sigma = 0.5 dip below
    min_norm somewhere on the grid), then normalised pointwise (assumption A3).
    """
    d = cfg.dim
    rng = np.random.Generator(np.random.PCG64(seed))
    rng_ks = [np.arange(-kmax, kmax + 1)] * d
    ks = np.stack(np.meshgrid(*rng_ks, indexing="ij"), -1).reshape(-1, d)
    norm2 = (ks ** 2).sum(1)
    ks = ks[(norm2 > 0) & (norm2 <= kmax * kmax)]
    amp = sigma / (1.0 + (ks ** 2).sum(1))
    # e^{2 pi i k x} per axis, k = -kmax..kmax: the field is the real part of a sum of
    # products of these (evaluated as d tensor contractions, not one cosine and one
    # sine per mode and grid point)
    xs = macro_coords(cfg)
    E = [np.exp(2j * math.pi * np.outer(np.arange(-kmax, kmax + 1), x)) for x in xs]
    shape = tuple(len(x) for x in xs)
    for attempt in range(128):
        if attempt and attempt % 16 == 0:
            amp = 0.7 * amp        # a field this rough keeps dipping below min_norm: make it smoother
        A = rng.standard_normal((3, len(ks)))
        B = rng.standard_normal((3, len(ks)))
        mt = np.empty((3,) + shape)
        for c in range(3):
            # A cos(2 pi k.x) + B sin(2 pi k.x) = Re((A - iB) e^{2 pi i k.x})
            Z = np.zeros((2 * kmax + 1,) * d, dtype=complex)
            Z[tuple((ks + kmax).T)] = amp * (A[c] - 1j * B[c])
            for a in range(d):
                Z = np.tensordot(Z, E[a], axes=([0], [0]))
            mt[c] = float(offset[c]) + Z.real
        nrm = np.sqrt((mt ** 2).sum(0))
        if nrm.min() >= min_norm:
            fourier_field.last_attempt = attempt
            return mt / nrm
    raise RuntimeError("fourier_field: could not draw a field with min |m| >= min_norm")


def ex1_initial(x: np.ndarray) -> np.ndarray:
    """(EX1) initial data of Section 2.4, normalised; x any shape -> (3, *x.shape)."""
    mt = np.stack([
        0.5 + np.exp(-0.1 * np.cos(2 * np.pi * (x - 0.32))),
        0.5 + np.exp(-0.2 * np.cos(2 * np.pi * x)),
        0.5 + np.exp(-0.1 * np.cos(2 * np.pi * (x - 0.75))),
    ])
    return mt / np.sqrt((mt ** 2).sum(0))


def ex2_initial_unnormalised(x1: np.ndarray, x2: np.ndarray) -> np.ndarray:
    """(EX2)/(EX3) m~ of Section 2.4 before normalisation."""
    c = np.cos
    tp = 2 * np.pi
    return np.stack([
        0.6 + np.exp(-0.3 * (c(tp * (x1 - 0.25)) + c(tp * (x2 - 0.12)))),
        0.5 + np.exp(-0.4 * (c(tp * x1) + c(tp * (x2 - 0.4)))),
        0.4 + np.exp(-0.2 * (c(tp * (x1 - 0.81)) + c(tp * (x2 - 0.73)))),
    ])


def ex2_initial(x1: np.ndarray, x2: np.ndarray) -> np.ndarray:
    """(EX2)/(EX3) initial data of Section 2.4, normalised."""
    mt = ex2_initial_unnormalised(x1, x2)
    return mt / np.sqrt((mt ** 2).sum(0))


def c1_initial(x: np.ndarray) -> np.ndarray:
    """1D benchmark initial data: normalised (0.5+0.3 sin 2pi x, 0.4 cos 2pi x, 0.6)."""
    mt = np.stack([0.5 + 0.3 * np.sin(2 * np.pi * x), 0.4 * np.cos(2 * np.pi * x),
                   np.full_like(x, 0.6)])
    return mt / np.sqrt((mt ** 2).sum(0))


def coeff_loc2d(X, eps):
    """The locally periodic 2D coefficient of Section 5 (eq. coeff_loc2D):
    0.25 exp(-cos(2 pi (x1 + x2)/eps) + sin(2 pi x1/eps) cos(2 pi x2))."""
    x1, x2 = X[0], X[1]
    tp = 2 * np.pi
    return 0.25 * np.exp(-np.cos(tp * (x1 + x2) / eps) + np.sin(tp * x1 / eps) * np.cos(tp * x2))


def face_table(cfg: HMMConfig) -> np.ndarray:
    """cfg.coef_fn tabulated at every face of every micro box, in the layout of
    hmm_set_face_table: boxes in macro-point order, per box d blocks of N^d values,
    block k at x_p + xi_j + (dx/2) e_k with xi_j = (j - (N-1)/2) dx, dx = eps_p/K
    (entries with j_k = N - 1 unused, set to 1)."""
    d = cfg.dim
    n = [int(v) for v in list(cfg.n_macro)[:d]]
    DX = [cfg.L / nk for nk in n]
    out = []
    for p in range(cfg.n_points):
        idx = np.unravel_index(p, n)
        eps = float(cfg.eps_field[p]) if cfg.eps_field is not None else float(cfg.eps)
        N = int(cfg.box_n_field[p]) if cfg.box_n_field is not None else int(cfg.box_n)
        dx = eps / cfg.pts_per_eps
        xi = (np.arange(N) - (N - 1) / 2.0) * dx
        for k in range(d):
            X = []
            for a in range(d):
                shp = [1] * d
                shp[a] = N
                X.append(idx[a] * DX[a] + (xi + (0.5 * dx if a == k else 0.0)).reshape(shp))
            vals = np.broadcast_to(np.asarray(cfg.coef_fn(X, eps), dtype=np.float64), (N,) * d).copy()
            last = [slice(None)] * d
            last[k] = N - 1
            vals[tuple(last)] = 1.0
            out.append(vals.ravel())
    return np.concatenate(out)


def uneven_eps_and_n(cfg: HMMConfig, K: float = 8.0, mu_prime: float = 0.015,
                     nmin: int = 32, nmax: int = 96, step: int = 8):
    """Locally varying eps and box sizes for the uneven-box workload.

    1/eps_i = 250 + 150 sin(2 pi x1) cos(2 pi x2) in [100, 400]; with K points
    per eps_i and a physical half-width mu' the box has
    N_i = clamp(step*ceil(2 mu' K/eps_i/step), nmin, nmax) nodes per axis.
    """
    X = _grid(cfg)
    inv = 250.0 + 150.0 * np.sin(2 * np.pi * X[0]) * np.cos(2 * np.pi * X[1])
    eps = 1.0 / inv
    n = step * np.ceil((2.0 * mu_prime * K / eps) / step)
    n = np.clip(n, nmin, nmax).astype(np.int32)
    return eps.reshape(-1).astype(np.float64), n.reshape(-1)


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------

def _sin(axis: int, scale: int = SCALE_FAST, omega: float = 1.0, phase: float = 0.0):
    return axis, KIND_SIN, scale, omega, phase


def _term(amp: float, *factors) -> CoefTerm:
    kind = [KIND_ONE] * 3
    scale = [SCALE_FAST] * 3
    omega = [1.0] * 3
    phase = [0.0] * 3
    for (ax, k, s, w, p) in factors:
        kind[ax], scale[ax], omega[ax], phase[ax] = k, s, w, p
    return CoefTerm(amp, tuple(kind), tuple(scale), tuple(omega), tuple(phase))


def _cos(axis: int, scale: int = SCALE_FAST, omega: float = 1.0, phase: float = 0.0):
    return axis, KIND_COS, scale, omega, phase


CONFIG_NAMES = ("c1_1d", "c2_2d", "c3_2d_uneven", "c4_3d", "c5_sweep")


def config(name: str, **over) -> HMMConfig:
    """Named workload configurations (sizes of the benchmark table).

    c1_1d         1D, 64 macro points, eps=1/100, a=1+0.5 sin(2 pi y), alpha=0.1,
                  N=201 (20 points per eps, width 10 eps), M=500, 4th-order stencil
    c2_2d         2D, 128^2 macro grid, eps=1/200, a=1+0.5 sin(2pi y1) sin(2pi y2),
                  alpha=0.05, N=64 (8 per eps), M=400
    c3_2d_uneven  2D, 256^2, a=1.1+0.25 sin(2pi y1)cos(2pi y2)+0.25 sin(2pi x1)sin(2pi y2),
                  eps_i in [1/400,1/100], N_i in 32..96, alpha=0.01, M=400, FP32 form
    c4_3d         3D, 64^3, eps=1/100, a=1+0.5 prod sin(2pi y_k), alpha=0.1, N=32
                  (6 per eps, mu=2 eps), M=300, FP32 form
    c5_sweep      2D laminated a=1+0.9 sin(2pi y1), eps=1/400, K=10 (sizes set per point)
    Micro damping alpha_micro = 1.2 (the paper's artificial damping) unless overridden.
    """
    if name == "c1_1d":
        cfg = HMMConfig(dim=1, n_macro=(64, 1, 1), alpha=0.1, alpha_micro=1.2,
                        c0=1.0, terms=[_term(0.5, _sin(0))], eps=1.0 / 100,
                        box_n=201, pts_per_eps=20.0, micro_steps=500, name=name)
    elif name == "c2_2d":
        cfg = HMMConfig(dim=2, n_macro=(128, 128, 1), alpha=0.05, alpha_micro=1.2,
                        c0=1.0, terms=[_term(0.5, _sin(0), _sin(1))], eps=1.0 / 200,
                        box_n=64, pts_per_eps=8.0, micro_steps=400, name=name)
    elif name == "c3_2d_uneven":
        cfg = HMMConfig(dim=2, n_macro=(256, 256, 1), alpha=0.01, alpha_micro=1.2,
                        c0=1.1, terms=[_term(0.25, _sin(0), _cos(1)),
                                       _term(0.25, _sin(0, SCALE_SLOW), _sin(1))],
                        eps=1.0 / 250, box_n=64, pts_per_eps=8.0, micro_steps=400,
                        precision=1, name=name)
    elif name == "c4_3d":
        cfg = HMMConfig(dim=3, n_macro=(64, 64, 64), alpha=0.1, alpha_micro=1.2,
                        c0=1.0, terms=[_term(0.5, _sin(0), _sin(1), _sin(2))],
                        eps=1.0 / 100, box_n=32, pts_per_eps=6.0, mu_over_eps=2.0,
                        micro_steps=300, precision=1, name=name)
    elif name == "c5_sweep":
        cfg = HMMConfig(dim=2, n_macro=(32, 32, 1), alpha=0.1, alpha_micro=1.0,
                        c0=1.0, terms=[_term(0.9, _sin(0))], eps=1.0 / 400,
                        box_n=64, pts_per_eps=10.0, micro_steps=400, name=name)
    elif name == "ex_loc2d":
        # Section 5, locally periodic 2D example: eq. coeff_loc2D, alpha = 0.1,
        # alpha_micro = 1.2, mu = 5 eps, mu' = 7 eps, eps = 0.01, (EX2) initial data,
        # DX = 1/16; K = 8 points per eps (not stated) gives N = 2 mu' K + 1 = 113.
        cfg = HMMConfig(dim=2, n_macro=(16, 16, 1), alpha=0.1, alpha_micro=1.2,
                        c0=1.0, terms=[], eps=0.01, box_n=113, pts_per_eps=8.0,
                        mu_over_eps=5.0, micro_steps=1250, coef_fn=coeff_loc2d, name=name)
    else:
        raise KeyError(name)
    cfg = dataclasses.replace(cfg, **over)
    if name == "c3_2d_uneven" and cfg.eps_field is None:
        eps, n = uneven_eps_and_n(cfg)
        cfg = dataclasses.replace(cfg, eps_field=eps, box_n_field=n)
    return cfg


def initial_field(cfg: HMMConfig, seed: Optional[int] = None) -> np.ndarray:
    """Seeded macro initial data M0 (3, P) for a named configuration."""
    if cfg.dim == 1:
        x = macro_coords(cfg)[0]
        m = c1_initial(x)
    elif cfg.name == "ex_loc2d":
        m = ex2_initial(*_grid(cfg))
    else:
        base = 20210820
        s = base + (CONFIG_NAMES.index(cfg.name) if cfg.name in CONFIG_NAMES else 7)
        m = fourier_field(cfg, s if seed is None else seed)
    return np.ascontiguousarray(m.reshape(3, -1))


# --------------------------------------------------------------------------
# Direct simulation resolving eps (the paper's reference solutions, Section 5)
# --------------------------------------------------------------------------


@dataclasses.dataclass
class DNSConfig:
    """Parameters of a direct simulation of eq. prob on a grid that resolves eps
    (the fields of the C struct hmm_dns_params).

    dim, n, L        periodic domain [0, L]^dim, n points per axis, dx = L/n
    alpha            damping (0 <= alpha <= 1)
    c0, terms, eps   a(x) = c0 + sum(terms), fast variable x/eps
    coef_fn          a coefficient that is not a sum of separable terms (tabulated
                     at the faces for the library); replaces c0 + terms when set
    dt, dt_safety    time step (<= 0: dt_safety times the MPEA stability step)
    stencil_order    2 or 4
    precision        0: FP64 state and arithmetic, 1: float-float state, FP32 arithmetic
    """
    dim: int
    n: Sequence[int]
    alpha: float
    c0: float
    terms: List[CoefTerm]
    eps: float
    L: float = 1.0
    dt: float = 0.0
    dt_safety: float = 0.5
    stencil_order: int = 4
    precision: int = 0
    coef_fn: Optional[Callable] = None
    name: str = ""

    @property
    def n_points(self) -> int:
        return int(np.prod([int(v) for v in list(self.n)[: self.dim]]))

    @property
    def shape(self):
        return tuple(int(v) for v in list(self.n)[: self.dim])

    def replace(self, **kw) -> "DNSConfig":
        return dataclasses.replace(self, **kw)


DNS_NAMES = ("dns_loc1d", "dns_quasi2d", "dns_loc2d")


def dns_config(name: str, **over) -> DNSConfig:
    """Named direct simulations of Section 5 (grid sizes as the paper states them).

    dns_loc1d    eq. loc: a = 1.1 + 0.25 sin(2 pi x + 1.1) + 0.5 sin(2 pi x/eps),
                 eps = 1/400, alpha = 0.01, dx = 1/6000 (15 points per eps)
    dns_quasi2d  eq. coeff_quasi: a = (1 + 0.25 sin(2 pi x1/eps))(1 + 0.25 sin(2 pi x2/eps)
                 + 0.25 sin(2 pi 1.41 x2/eps)), expanded into six separable terms,
                 eps = 0.01, alpha = 0.01, dx = 1/1500
    dns_loc2d    eq. coeff_loc2D (tabulated), eps = 0.01, alpha = 0.1; the paper does
                 not state its dx; 15 points per eps as in the other two (dx = 1/1500)
    """
    if name == "dns_loc1d":
        cfg = DNSConfig(dim=1, n=(6000, 1, 1), alpha=0.01, c0=1.1,
                        terms=[_term(0.25, _sin(0, SCALE_SLOW, 1.0, 1.1)), _term(0.5, _sin(0))],
                        eps=1.0 / 400, name=name)
    elif name == "dns_quasi2d":
        r = 1.41
        cfg = DNSConfig(dim=2, n=(1500, 1500, 1), alpha=0.01, c0=1.0,
                        terms=[_term(0.25, _sin(1)), _term(0.25, _sin(1, omega=r)),
                               _term(0.25, _sin(0)), _term(0.0625, _sin(0), _sin(1)),
                               _term(0.0625, _sin(0), _sin(1, omega=r))],
                        eps=0.01, name=name)
    elif name == "dns_loc2d":
        cfg = DNSConfig(dim=2, n=(1500, 1500, 1), alpha=0.1, c0=1.0, terms=[], eps=0.01,
                        coef_fn=coeff_loc2d, name=name)
    else:
        raise KeyError(name)
    return dataclasses.replace(cfg, **over)


def dns_coords(cfg: DNSConfig) -> List[np.ndarray]:
    """Grid nodes x_j = j L/n per axis."""
    return [np.arange(n) * (cfg.L / n) for n in cfg.shape]


def dns_initial(cfg: DNSConfig, noise: float = 0.0, seed: int = 20210820) -> np.ndarray:
    """Initial data (3, prod n) on the grid: (EX1) in 1D, (EX2) in 2D, as in the
    paper's direct simulations; ``noise`` > 0 adds seeded N(0, noise^2) values to
    every component before normalisation (rough data for parity tests)."""
    X = np.meshgrid(*dns_coords(cfg), indexing="ij")
    if cfg.dim == 1:
        mt = ex1_initial(X[0])
    elif cfg.dim == 2:
        mt = ex2_initial_unnormalised(X[0], X[1])
    else:
        raise ValueError("direct simulations are defined for d = 1 and 2")
    if noise > 0:
        rng = np.random.Generator(np.random.PCG64(seed))
        mt = mt + noise * rng.standard_normal(mt.shape)
    m = mt / np.sqrt((mt ** 2).sum(0))
    return np.ascontiguousarray(m.reshape(3, -1))
