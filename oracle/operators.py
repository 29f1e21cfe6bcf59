"""Radial operators in coefficient space (oracle, FP64).

del2h_closed(m, nc, ell)
    Matrix of the horizontal Laplacian D_m on the normalised coefficients,
    built from the pentadiagonal entries of Eq. (5) (which act on the
    unnormalised P_n^m and scale as ell^-2), rescaled to the orthonormal basis by
    N_j / N_n for entry (n, j) (Sec. 3.1, below Eq. (7); the paper writes it as
    exp(ln N_j - ln N_n), evaluated here as the exact factorial ratio).
    Row n is the output degree, column j the input degree; entries beyond the
    chop Nc are dropped (truncation).

del2h_quadrature(m, nc, ell)
    Independent construction.  Dividing the mapped Legendre equation Eq. (3) by r
    gives grad_h^2 P_{ell,n}^m = -n(n+1) (1-x)^2 ell^-2 P_{ell,n}^m, hence
        D_m[n, j] = -j(j+1)/ell^2 * int (1-x)^2 Pbar_n^m Pbar_j^m dx,
    evaluated with Nc + 2 Gauss nodes (exact: the integrand has degree <= 2 Nc).

rdr_matrix(m, nc)
    r d/dr = (1 - x^2) d/dx under Eq. (1).  With the Ferrers identities
    (1-x^2) dP_n^m/dx = (n+m) P_{n-1}^m - n x P_n^m and
    (2n+1) x P_n^m = (n-m+1) P_{n+1}^m + (n+m) P_{n-1}^m:
        r d/dr P_n^m = (n+1)(n+m)/(2n+1) P_{n-1}^m - n(n-m+1)/(2n+1) P_{n+1}^m,
    i.e. tridiagonal (Sec. 3.1), then rescaled to the orthonormal basis.

linear_operator(m, kappa, nc, ell, nu, nu_h, p)
    Eq. (11) on harmonic (m, k): L = nu (D_m - kappa^2 I) - nu_h (-(D_m - kappa^2 I))^{p/2}
    (Eq. (4) for the full Laplacian).  The power is a product of the truncated
    (Nc-m) x (Nc-m) matrices ("shifting and composing", Sec. 3.1; truncate then
    compose is the reading taken).

Pins: the two Laplacian constructions agree; the hand closed form
ell^2 lap P_1^0 = 4/3 P_0 - 16/5 P_1 + 8/3 P_2 - 4/5 P_3; spectral derivative of
analytic fields; exact decay of closed-form diffusion solutions (Sec. 5.1).
"""

from fractions import Fraction
import functools
import math

import numpy as np

from .basis import pbar_table
from .grid import gauss_legendre


def norm_ratio(j, n, m):
    """N_j^m / N_n^m of Eq. (7), from the exact factorial ratio, correctly rounded.

    (exp(ln N_j - ln N_n) with rounded logs of size ~n log n carries ~1e-14
    relative error at n ~ 100; the exact ratio does not.)
    """
    m = abs(m)
    q = Fraction((2 * j + 1) * math.factorial(j - m) * math.factorial(n + m),
                 (2 * n + 1) * math.factorial(n - m) * math.factorial(j + m))
    return math.sqrt(q)


def _rescale(Mat, m, nc):
    """Entry (row a, col b) (degrees n = m + a, j = m + b) times N_j / N_n."""
    out = Mat.copy()
    rows, cols = np.nonzero(Mat)
    for a, b in zip(rows, cols):
        out[a, b] = Mat[a, b] * norm_ratio(m + int(b), m + int(a), m)
    return out


def del2h_unnormalised(m, nc, ell):
    """Eq. (5): D[n, j] on unnormalised coefficients, n, j in [m, nc)."""
    m = abs(m)
    N = nc - m
    D = np.zeros((N, N))
    for n in range(m, nc):
        a = n - m
        if n - 2 >= m:
            D[a, a - 2] = -((n - m - 1) * (n - m) * (n - 2) * (n - 1)) / ((2 * n - 3) * (2 * n - 1))
        if n - 1 >= m:
            D[a, a - 1] = 2.0 * n * (n - 1) * (n - m) / (2 * n - 1)
        D[a, a] = -2.0 * n * (n + 1) * (3 * n * n + 3 * n - m * m - 2) / ((2 * n - 1) * (2 * n + 3))
        if n + 1 < nc:
            D[a, a + 1] = 2.0 * (n + 1) * (n + 2) * (n + m + 1) / (2 * n + 3)
        if n + 2 < nc:
            D[a, a + 2] = -((n + 2) * (n + 3) * (n + m + 1) * (n + m + 2)) / ((2 * n + 3) * (2 * n + 5))
    return D / (ell * ell)


@functools.lru_cache(maxsize=4096)
def _del2h_closed_cached(m, nc, ell):
    return _rescale(del2h_unnormalised(m, nc, ell), m, nc)


def del2h_closed(m, nc, ell):
    """D_m on the orthonormal coefficients (a fresh copy; the exact rescaling is
    computed once per (m, Nc, ell) and reused, since it does not depend on kappa)."""
    return _del2h_closed_cached(abs(int(m)), int(nc), float(ell)).copy()


def del2h_quadrature(m, nc, ell):
    m = abs(m)
    xq, wq = gauss_legendre(nc + 2)
    P = pbar_table(m + 1, nc, xq)[m]                     # [nc-m][nq]
    G = (P * (wq * (1.0 - xq) ** 2)[None, :]) @ P.T      # <Pbar_n (1-x)^2 Pbar_j>
    j = np.arange(m, nc, dtype=np.float64)
    return G * (-(j * (j + 1.0)) / (ell * ell))[None, :]


def rdr_matrix(m, nc):
    """(r d/dr) on normalised coefficients of order m: out[j] = sum_n R[j, n] in[n]."""
    m = abs(m)
    N = nc - m
    R = np.zeros((N, N))
    for n in range(m, nc):
        a = n - m
        if n - 1 >= m:
            R[a - 1, a] = (n + 1.0) * (n + m) / (2 * n + 1)
        if n + 1 < nc:
            R[a + 1, a] = -n * (n - m + 1.0) / (2 * n + 1)
    # unnormalised coefficient c_n = N_n cbar_n; out_bar[j] = out[j] / N_j,
    # i.e. entry (row j, col n) times N_n / N_j
    return _rescale(R, m, nc)


def linear_operator(m, kappa, nc, ell, nu, nu_h=0.0, p=8):
    D = del2h_closed(m, nc, ell)
    lap = D - kappa * kappa * np.eye(D.shape[0])
    L = nu * lap
    if nu_h != 0.0:
        if p not in (4, 6, 8):
            raise ValueError("hyperviscosity power p must be 4, 6 or 8 (Eq. (11))")
        neg = -lap
        pw = np.eye(D.shape[0])
        for _ in range(p // 2):
            pw = pw @ neg
        L = L - nu_h * pw
    return L


def logproxy_image(ell):
    """Eq. (6): coefficients of grad_h^2 ln(r^2 + ell^2) on unnormalised P_0^0..P_2^0."""
    return np.array([4.0 / 3.0, -2.0, 2.0 / 3.0]) / (ell * ell)

