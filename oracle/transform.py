"""Spectral transform pair of the truncated expansion Eq. (2) (oracle, FP64).

Backward (spectral -> physical), straight from Eq. (2) for a real scalar:
    f_mk(r_i)  = sum_{n=m}^{Nc-1} shat_nmk Pbar_n^m(x_i)
    s(r,phi,z) = sum_k f_0k e^{i kappa_k z}  +  2 Re sum_{m>=1} sum_k f_mk e^{i(m phi + kappa_k z)}
(only m >= 0 is stored since shat_{n,-m,-k} = conj(shat_nmk); the real part of
the m = 0 sum is taken).

Forward (physical -> spectral): the naive DFTs with 1/Nphi and 1/Nz, then Gauss
quadrature against the orthonormal basis:
    shat_nmk = sum_i w_i Pbar_n^m(x_i) f_mk(r_i).
When the chop keeps the Nyquist index (|m| = Nphi/2, or |k| = Nz/2), the two
members of the pair (+N/2, -N/2) multiply the same grid function (-1)^j, so the
grid fixes only their sum.  The paper does not say how the sum is shared; the
reading taken is the minimum-norm one, equal halves: the Nyquist DFT row carries
a factor 1/2 in the forward direction, and the backward direction is Eq. (2)
summed over both members as written (the m = Nphi/2 term enters with the factor
2 of every m >= 1, the rows k = +Nz/2 and k = -Nz/2 are both summed).
The DFTs are explicit matrices with phases 2 pi ((j m) mod N) / N (integer-reduced
angle), applied with a library matmul.  The radial step is the dense triangular
quadrature per m (the paper's Sec. 4.1 calls it a banded product along r; only
the operators are banded, so it is read as dense).

Spectral storage: a list over m of complex arrays [K][Nc - m] (k in FFT order).
to_flat/from_flat map that list to the flat ragged layout
    index(m, k, n) = K * sum_{m' < m} (Nc - m') + k * (Nc - m) + (n - m)
with complex128 entries, the layout of the library's spectral buffers.

Pins: round-trip identity spectral -> physical -> spectral, numpy.fft, azimuthal
purity (Sec. 5.1), representation errors of Sec. 5.1.
"""

import contextlib
import math

import numpy as np


def serial():
    """Context in which the BLAS/LAPACK calls run on one thread.  The oracle's
    per-harmonic loops apply many small (<= 1024 x 1024) dense operations, for
    which a multithreaded BLAS is slower than one thread; the arithmetic is the
    same either way."""
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:          # pragma: no cover - threadpoolctl ships with scikit-learn
        return contextlib.nullcontext()
    return threadpool_limits(1)


def _dft_matrix(nout_idx, npts, sign):
    """E[a, j] = exp(sign * 2 pi i ((idx_a * j) mod N) / N)."""
    j = np.arange(npts, dtype=np.int64)
    ph = (np.asarray(nout_idx, dtype=np.int64)[:, None] * j[None, :]) % npts
    ang = 2.0 * math.pi * ph / npts
    return np.cos(ang) + sign * 1j * np.sin(ang)


def spec_zeros(g):
    return [np.zeros((g.K, g.nc - m), dtype=np.complex128) for m in range(g.M)]


def forward(g, phys):
    """phys: real [Nz][Nphi][Nr] -> list of [K][Nc-m] complex."""
    phys = np.asarray(phys, dtype=np.float64)
    assert phys.shape == (g.nz, g.nphi, g.nr)
    Ephi = _dft_matrix(np.arange(g.M), g.nphi, -1.0) / g.nphi       # [M][Nphi]
    if g.nphi >= 2 and g.M - 1 == g.nphi // 2:
        Ephi[g.M - 1] *= 0.5                                           # m = +-Nphi/2 halves
    f1 = np.einsum("mj,zji->zmi", Ephi, phys)                         # [Nz][M][Nr]
    Ez = _dft_matrix(g.kz, g.nz, -1.0) / g.nz                          # [K][Nz]
    if g.nz > 1:
        Ez[np.abs(g.kz) == g.nz // 2] *= 0.5                           # k = +-Nz/2 halves
    f2 = np.einsum("kz,zmi->kmi", Ez, f1)                              # [K][M][Nr]
    out = []
    for m in range(g.M):
        Wm = g.P[m] * g.w[None, :]                                     # [Nc-m][Nr]
        out.append(f2[:, m, :] @ Wm.T)                                 # [K][Nc-m]
    return out


def backward(g, spec):
    """list of [K][Nc-m] complex -> real [Nz][Nphi][Nr]."""
    f2 = np.zeros((g.K, g.M, g.nr), dtype=np.complex128)
    for m in range(g.M):
        f2[:, m, :] = spec[m] @ g.P[m]
    Ez = _dft_matrix(g.kz, g.nz, 1.0).T                                # [Nz][K]
    f1 = np.einsum("zk,kmi->zmi", Ez, f2)                              # [Nz][M][Nr]
    Ephi = _dft_matrix(np.arange(g.M), g.nphi, 1.0).T                 # [Nphi][M]
    mult = np.full(g.M, 2.0)
    mult[0] = 1.0
    phys = np.einsum("jm,zmi->zji", Ephi * mult[None, :], f1).real
    return phys


def offsets(g):
    off = [0]
    for m in range(g.M):
        off.append(off[-1] + g.K * (g.nc - m))
    return off


def to_flat(g, spec):
    off = offsets(g)
    flat = np.zeros(off[-1], dtype=np.complex128)
    for m in range(g.M):
        flat[off[m]:off[m + 1]] = spec[m].reshape(-1)
    return flat


def from_flat(g, flat):
    off = offsets(g)
    flat = np.asarray(flat)
    if flat.dtype != np.complex128:
        flat = flat.view(np.complex128) if flat.dtype == np.float64 else flat.astype(np.complex128)
    return [flat[off[m]:off[m + 1]].reshape(g.K, g.nc - m).copy() for m in range(g.M)]


def spec_norm(g, spec):
    """Spectral l2 norm with multiplicity 2 for m >= 1 (the real field's Parseval weight)."""
    tot = 0.0
    for m in range(g.M):
        tot += (1.0 if m == 0 else 2.0) * float(np.sum(np.abs(spec[m]) ** 2))
    return math.sqrt(tot)


def spec_rel_err(g, a, b):
    """||a - b|| / ||b|| in the spectral norm above."""
    d = [a[m] - b[m] for m in range(g.M)]
    nb = spec_norm(g, b)
    return spec_norm(g, d) / (nb if nb > 0 else 1.0)
