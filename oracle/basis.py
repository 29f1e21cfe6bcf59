"""Normalised associated Legendre functions (oracle, FP64).

Pbar_n^m = N_n^m P_n^m with N_n^m = sqrt((2n+1)(n-m)! / (2 (n+m)!))  (Eq. (7)),
so that int_{-1}^{1} Pbar_n^m Pbar_{n'}^m dx = delta_{nn'}.  The paper leaves the
Condon-Shortley phase unstated; no phase is used (P_m^m = (2m-1)!! (1-x^2)^{m/2} > 0).

Evaluation: the order-m diagonal Pbar_m^m is climbed from Pbar_0^0 = 1/sqrt(2) by
Pbar_m^m = sqrt((2m+1)/(2m)) sqrt(1-x^2) Pbar_{m-1}^{m-1}, then the degree is raised
by the normalised three-term recurrence obtained by dividing
(n-m) P_n^m = (2n-1) x P_{n-1}^m - (n+m-1) P_{n-2}^m by N_n^m.  No factorial is
ever formed (Sec. 3.1 explains why the factorials cannot be used in FP64).

ln_norm returns ln N_n^m through lgamma, used only by the closed-form operator
rescaling (Sec. 3.1) and by the tests.

Pins: discrete orthonormality under the Gauss rule, scipy.special.lpmv times
exp(ln N) (up to the (-1)^m phase lpmv carries).
"""

import math

import numpy as np


def ln_norm(n, m):
    """ln N_n^m of Eq. (7) via lgamma."""
    m = abs(m)
    return 0.5 * (math.log(2 * n + 1) + math.lgamma(n - m + 1) - math.log(2.0)
                  - math.lgamma(n + m + 1))


def pbar_table(M, nc, x):
    """List over m < M of arrays [nc - m][len(x)] with Pbar_n^m(x_i), n = m..nc-1."""
    x = np.asarray(x, dtype=np.float64)
    s = np.sqrt((1.0 - x) * (1.0 + x))
    out = []
    pmm = np.full_like(x, 1.0 / math.sqrt(2.0))
    for m in range(M):
        if m > 0:
            pmm = math.sqrt((2 * m + 1) / (2.0 * m)) * s * pmm
        tab = np.zeros((nc - m, x.size))
        tab[0] = pmm
        if nc - m > 1:
            tab[1] = math.sqrt(2 * m + 3) * x * pmm
        for n in range(m + 2, nc):
            a = math.sqrt((4.0 * n * n - 1.0) / (n * n - m * m))
            b = math.sqrt(((n - 1.0) ** 2 - m * m) / (4.0 * (n - 1.0) ** 2 - 1.0))
            tab[n - m] = a * (x * tab[n - m - 1] - b * tab[n - m - 2])
        out.append(tab)
    return out
