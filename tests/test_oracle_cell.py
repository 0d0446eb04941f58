"""Pins of the oracle's homogenised-coefficient solver (Section 2.1, eqs. AH, cell_problem).

Closed forms (1D harmonic mean, laminated diag(harmonic, arithmetic), the
separable (EX3) value 1.1 sqrt(1.1^2 - 0.25)) and the printed (EX2) matrix
(Section 2.4, 3 decimals) fix the solver that supplies A^H to other tests.
"""
import json
import os

import numpy as np

from oracle import cell_problem as C

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "homogenised_coefficients.json")))
tp = 2 * np.pi


def test_1d_harmonic_mean_ex1():
    ah = C.homogenised_coefficient_1d(lambda y: 1 + 0.5 * np.sin(tp * y))
    assert abs(ah - np.sqrt(0.75)) < 1e-13
    assert abs(ah - GOLD["EX1"]["AH"]) < 5e-4


def test_laminated():
    AH = C.homogenised_coefficient_2d(lambda y1, y2: 1 + 0.9 * np.sin(tp * y1) + 0 * y2, 64)
    np.testing.assert_allclose(AH, np.diag([np.sqrt(0.19), 1.0]), atol=1e-9)


def test_ex3_closed_form():
    AH = C.homogenised_coefficient_2d(
        lambda y1, y2: (1.1 + 0.5 * np.sin(tp * y1)) * (1.1 + 0.5 * np.sin(tp * y2)), 64)
    np.testing.assert_allclose(AH, 1.1 * np.sqrt(1.1 ** 2 - 0.25) * np.eye(2), atol=1e-7)


def test_ex2_printed_values():
    a = lambda y1, y2: (0.5 + (0.5 + 0.25 * np.sin(tp * y1)) * (0.5 + 0.25 * np.sin(tp * y2))
                        + 0.25 * (np.cos(tp * (y1 - y2)) + np.sin(tp * y1)))
    AH = C.homogenised_coefficient_2d(a, 64)
    np.testing.assert_allclose(AH, np.array(GOLD["EX2"]["AH"]), atol=5e-4)
    assert abs(AH[0, 1] - AH[1, 0]) < 1e-10
