"""Analysis of measured diagnostics (not part of the transform method): the Crow
instability's theoretical growth rate and the fitted rate of a measured modal
energy history (Sec. 5.3).

crow_alpha(beta, a_over_b) evaluates Crow's dispersion relation for the symmetric
mode of a counter-rotating pair (Eq. (crow-dispersion) of the paper),
    alpha_S^2 = (1 - eta + beta^2 varpi)(1 + xi - beta^2 varpi),
    xi = beta K1(beta), eta = beta^2 K0(beta) + beta K1(beta),
    varpi(delta) = (1/2) [(cos delta - 1)/delta^2 + sin delta / delta - Ci(delta)],
with beta = kappa b, delta = kappa d and the Lamb-Oseen cut-off distance
d = a exp((1 - gamma_E - ln 2) / 2) ~ 0.8736 a; alpha is in units of Gamma / (2 pi b^2).
growth_rate(t, E, b, gamma) fits alpha = (pi b^2 / Gamma) d ln E / dt by least squares.
"""

import math

import numpy as np


def crow_cutoff(a):
    """Crow's cut-off distance of a Lamb-Oseen core of radius a."""
    return a * math.exp((1.0 - np.euler_gamma - math.log(2.0)) / 2.0)


def crow_alpha(beta, a_over_b):
    import scipy.special as sp
    delta = beta * crow_cutoff(a_over_b)          # kappa d with b = 1
    xi = beta * sp.k1(beta)
    eta = beta * beta * sp.k0(beta) + beta * sp.k1(beta)
    ci = sp.sici(delta)[1]
    varpi = 0.5 * ((math.cos(delta) - 1.0) / delta ** 2 + math.sin(delta) / delta - ci)
    a2 = (1.0 - eta + beta * beta * varpi) * (1.0 + xi - beta * beta * varpi)
    return math.sqrt(a2) if a2 > 0 else 0.0


def growth_rate(t, E, b, gamma, window):
    """alpha = (pi b^2 / Gamma) d ln E / dt, least-squares slope over t in window."""
    t = np.asarray(t, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    sel = (t >= window[0]) & (t <= window[1]) & (E > 0)
    if np.count_nonzero(sel) < 3:
        return None
    slope = np.polyfit(t[sel], np.log(E[sel]), 1)[0]
    return math.pi * b * b / gamma * slope
