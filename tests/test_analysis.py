"""CPU checks of the analysis helpers (Crow dispersion relation, rate fit)."""

import math

import numpy as np

from paper_2609_18026_b300 import analysis as A


def test_crow_theory_matches_paper_value():
    # Sec. 5.3: at beta = 0.7306 and a / b = 0.125 (Lamb-Oseen cut-off d = 0.8736 a)
    # the dispersion relation predicts alpha_theory = 0.798
    assert abs(A.crow_cutoff(1.0) - 0.8736) < 5e-5
    assert abs(A.crow_alpha(2 * math.pi / 8.6, 0.125) - 0.798) < 5e-4


def test_growth_rate_fit():
    t = np.linspace(0, 20, 81)
    b, gamma = 4.0, 2 * math.pi
    alpha = 0.8
    sigma = alpha * gamma / (2 * math.pi * b * b)     # amplitude rate in physical units
    E = 1e-6 * np.exp(2 * sigma * t)                 # energy grows at twice the amplitude rate
    assert abs(A.growth_rate(t, E, b, gamma, (5, 15)) - alpha) < 1e-9
