"""Homogenised coefficient A^H from the periodic cell problem (oracle validator).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). Used to give the target
div(grad m A^H) that H_avg approximates (Section 2.2, Theorem 2) for
coefficients without a closed-form A^H.

A^H = int_Y a (I + (grad chi)^T) dy with div(a grad chi_k) = -d_k a, chi_k of
zero mean (Section 2.1, eqs. AH and cell_problem). Discretised by the
conservative 5-point scheme on an n^d periodic grid with a at the faces; in
that discretisation A^H_kl equals the discrete energy form
sum_faces a (e_k + D chi_k).(e_l + D chi_l) / n^d, which is second order in 1/n;
Richardson extrapolation over n and 2n removes the leading term.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _cell_AH_2d(a_fun, n: int) -> np.ndarray:
    h = 1.0 / n
    y = np.arange(n) * h
    Y1, Y2 = np.meshgrid(y, y, indexing="ij")
    ax = a_fun(Y1 + 0.5 * h, Y2)       # face between (i, j) and (i+1, j)
    ay = a_fun(Y1, Y2 + 0.5 * h)       # face between (i, j) and (i, j+1)
    N = n * n
    idx = np.arange(N).reshape(n, n)
    ip = np.roll(idx, -1, 0)
    jp = np.roll(idx, -1, 1)
    rows, cols, vals = [], [], []
    for (nb, af) in ((ip, ax), (jp, ay)):
        a_ = af.ravel()
        i0, i1 = idx.ravel(), nb.ravel()
        # energy a (u_i1 - u_i0)^2 -> stiffness contributions
        rows += [i0, i1, i0, i1]
        cols += [i0, i1, i1, i0]
        vals += [a_, a_, -a_, -a_]
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    # The stiffness matrix is A u = -h^2 div_h(a grad_h u); the cell problem
    # div_h(a (grad_h chi_k + e_k)) = 0 gives A chi_k = h^2 div_h(a e_k).
    b1 = (ax - np.roll(ax, 1, 0)) * h
    b2 = (ay - np.roll(ay, 1, 1)) * h
    # pin one node (zero-mean solution recovered afterwards)
    A = A.tolil()
    A[0, :] = 0
    A[0, 0] = 1.0
    A = A.tocsc()
    chis = []
    for b in (b1, b2):
        rhs = b.ravel().copy()
        rhs[0] = 0.0
        chi = spla.spsolve(A, rhs).reshape(n, n)
        chis.append(chi - chi.mean())
    # discrete gradients at faces (units: chi is in length units)
    AH = np.zeros((2, 2))
    Dx = [(np.roll(c, -1, 0) - c) / h for c in chis]
    Dy = [(np.roll(c, -1, 1) - c) / h for c in chis]
    for k in range(2):
        for l in range(2):
            ex = (1.0 if k == 0 else 0.0) + Dx[k]
            ex2 = (1.0 if l == 0 else 0.0) + Dx[l]
            ey = (1.0 if k == 1 else 0.0) + Dy[k]
            ey2 = (1.0 if l == 1 else 0.0) + Dy[l]
            AH[k, l] = (ax * ex * ex2).mean() + (ay * ey * ey2).mean()
    return AH


def homogenised_coefficient_2d(a_fun, n: int = 128) -> np.ndarray:
    """A^H for a 1-periodic a(y1, y2), Richardson-extrapolated from n and 2n."""
    A1 = _cell_AH_2d(a_fun, n)
    A2 = _cell_AH_2d(a_fun, 2 * n)
    return (4.0 * A2 - A1) / 3.0


def homogenised_coefficient_1d(a_fun, n: int = 4096) -> float:
    """A^H in 1D from the same conservative discretisation (a discrete harmonic mean)."""
    y = (np.arange(n) + 0.5) / n
    return 1.0 / np.mean(1.0 / a_fun(y))
