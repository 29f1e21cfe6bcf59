"""Collocation grid of the mapped Legendre / Fourier method (oracle, FP64).

* Radial: Gauss-Legendre nodes x_i on (-1, 1) (Sec. 3.1), mapped to
  r_i = ell * sqrt((1 + x_i) / (1 - x_i))   (Eq. (1)).
* Azimuthal: phi_j = 2 pi j / Nphi; axial: z_l = Lz l / Nz, both starting at 0
  (the paper does not state an offset; zero is the reading taken).
* Chops (Sec. 3.1, Eq. (2)): m = 0..M-1 stored (M = Nphi^c), k in FFT order
  0..Kz-1, -(Kz-1)..-1 (K = 2 Kz - 1 stored wavenumbers), n = m..Nc-1.
  Policies: "linear" keeps M = Nphi/2, Kz = max(1, Nz/2) (Nyquist dropped);
  "twothirds" keeps M = (Nphi-1)//3 + 1, Kz = (Nz-1)//3 + 1 (the two-thirds
  mask of Sec. 3.3 realised as storage truncation); "nyquist" keeps
  |m| <= Nphi/2 and |k| <= Nz/2 (M = Nphi/2 + 1, Kz = Nz/2 + 1, or 1 when
  Nz = 1), the |m| <= 128, |k| <= 128 layout of the 256^3 production run of
  Sec. 4.2; Nc = Nr unless given.  With the Nyquist kept, the pairs m = +-Nphi/2
  and k = +-Nz/2 coincide on the grid; see transform.py for how they are split.

Pins: numpy.polynomial.legendre.leggauss, exact integration of x^k, half the
nodes inside r < ell (Sec. 3.1), outermost node 20.36 ell at Nr = 24 (Sec. 1).
"""

import math

import numpy as np


def _legendre_pair(n, x):
    """P_n(x) and P_{n-1}(x) by the Bonnet three-term recurrence."""
    p0 = np.ones_like(x)
    if n == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    for k in range(2, n + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    return p1, p0


def gauss_legendre(n):
    """n-point Gauss-Legendre nodes (ascending) and weights on (-1, 1).

    Newton iteration on P_n from the Chebyshev-like initial guesses; weights
    w_i = 2 / ((1 - x_i^2) P_n'(x_i)^2).
    """
    i = np.arange(1, n + 1, dtype=np.float64)
    x = np.cos(np.pi * (i - 0.25) / (n + 0.5))
    for _ in range(100):
        pn, pm1 = _legendre_pair(n, x)
        dp = -n * (x * pn - pm1) / ((1.0 - x) * (1.0 + x))
        dx = pn / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    pn, pm1 = _legendre_pair(n, x)
    dp = -n * (x * pn - pm1) / ((1.0 - x) * (1.0 + x))
    w = 2.0 / ((1.0 - x) * (1.0 + x) * dp * dp)
    order = np.argsort(x)
    return x[order], w[order]


def map_r(x, ell):
    """Eq. (1): r = ell sqrt((1+x)/(1-x))."""
    return ell * np.sqrt((1.0 + x) / (1.0 - x))


def chops(nphi, nz, policy):
    if policy == "linear":
        M = max(1, nphi // 2)
        Kz = max(1, nz // 2)
    elif policy == "twothirds":
        M = (nphi - 1) // 3 + 1
        Kz = (nz - 1) // 3 + 1
    elif policy == "nyquist":
        M = nphi // 2 + 1
        Kz = nz // 2 + 1 if nz > 1 else 1
    else:
        raise ValueError(policy)
    return M, Kz


class Grid:
    """Nodes, weights, basis tables and wavenumbers for one (Nr, Nphi, Nz, ell, Lz)."""

    def __init__(self, nr, nphi, nz, ell, lz=2.0 * math.pi, policy="linear",
                 nr_c=None, M=None, Kz=None):
        from .basis import pbar_table
        self.nr, self.nphi, self.nz = nr, nphi, nz
        self.ell, self.lz = float(ell), float(lz)
        M0, Kz0 = chops(nphi, nz, policy)
        self.M = M if M is not None else M0
        self.Kz = Kz if Kz is not None else Kz0
        self.K = 2 * self.Kz - 1
        self.nc = nr if nr_c is None else nr_c
        if self.M > self.nc:
            raise ValueError("azimuthal chop exceeds radial chop")
        self.x, self.w = gauss_legendre(nr)
        self.r = map_r(self.x, self.ell)
        self.phi = 2.0 * math.pi * np.arange(nphi) / nphi
        self.zz = self.lz * np.arange(nz) / nz
        self.kz = np.array([k if k < self.Kz else k - self.K for k in range(self.K)],
                           dtype=np.int64)
        self.kappa = 2.0 * math.pi * self.kz / self.lz
        # P[m] has shape [Nc - m][Nr]: P[m][n - m, i] = Pbar_n^m(x_i)
        self.P = pbar_table(self.M, self.nc, self.x)

    def nodes3(self):
        """Broadcastable (r, phi, z) arrays in the physical layout [Nz][Nphi][Nr]."""
        return (self.r[None, None, :], self.phi[None, :, None], self.zz[:, None, None])
