"""Coefficients given as functions and tabulated at the faces (hmm_set_face_table).

CPU checks of the host-side logic: the oracle evaluates a coefficient function
exactly where it evaluates the separable terms, and the face table laid out for
the library holds, block by block, the oracle's face coefficients of each box.
"""
import numpy as np

import workloads as W
from oracle import hmm_oracle as O


def _as_function(cfg):
    """The c2 coefficient 1 + 0.5 sin(2 pi y1) sin(2 pi y2) written as a function."""
    def a(X, eps):
        tp = 2 * np.pi
        return 1.0 + 0.5 * np.sin(tp * X[0] / eps) * np.sin(tp * X[1] / eps)
    return cfg.replace(coef_fn=a)


def test_coefficient_function_matches_terms():
    cfg = W.config("c2_2d", n_macro=(8, 8, 1), box_n=24, micro_steps=10)
    cfn = _as_function(cfg)
    for p in (0, 9, 63):
        geo = O.box_geometry(cfg, p)
        for ft, ff in zip(O.face_coefficients(cfg, geo), O.face_coefficients(cfn, geo)):
            assert np.abs(ft - ff).max() < 1e-12   # sin arguments up to 2 pi x/eps ~ 300 rounded differently
        # the micro step follows the box's own maximum, at most the bound c0 + sum |amp|
        assert O.box_geometry(cfn, p)["dt"] >= geo["dt"] * (1 - 1e-15)


def test_face_table_layout_matches_oracle_faces():
    cfg = W.config("ex_loc2d", n_macro=(6, 5, 1), box_n=21, micro_steps=10)
    tab = W.face_table(cfg)
    N, d = cfg.box_n, cfg.dim
    assert tab.size == cfg.n_points * d * N ** d
    for p in (0, 7, cfg.n_points - 1):
        geo = O.box_geometry(cfg, p)
        faces = O.face_coefficients(cfg, geo)
        for k in range(d):
            blk = tab[(p * d + k) * N ** d:(p * d + k + 1) * N ** d].reshape((N,) * d)
            used = [slice(None)] * d
            used[k] = slice(0, N - 1)
            assert np.abs(blk[tuple(used)] - faces[k]).max() <= 1e-12 * np.abs(faces[k]).max()


def test_locally_periodic_coefficient_positive_and_bounded():
    """(A1): eq. coeff_loc2D lies in [0.25 e^-2, 0.25 e^2]."""
    x = np.random.default_rng(0).random((2, 10000))
    a = W.coeff_loc2d([x[0], x[1]], 0.01)
    assert a.min() >= 0.25 * np.exp(-2) * (1 - 1e-12) and a.max() <= 0.25 * np.exp(2) * (1 + 1e-12)
