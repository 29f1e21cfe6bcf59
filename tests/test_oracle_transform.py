"""Pins of the oracle's transform pair (CPU only)."""

import json
import math
import os

import numpy as np
import pytest
import scipy.special as sp

import oracle as O
from paper_2609_18026_b300 import workloads as W


def _rand_spec(g, seed):
    flat = W.random_spectral(g.nc, g.M, g.Kz, seed=seed)
    return O.from_flat(g, flat)


@pytest.mark.parametrize("nr,nphi,nz,policy", [
    (4, 4, 1, "linear"), (6, 8, 4, "linear"), (8, 8, 4, "twothirds"),
    (17, 12, 6, "linear"), (32, 16, 8, "twothirds"), (48, 32, 16, "linear")])
def test_roundtrip_spectral_identity(nr, nphi, nz, policy):
    g = O.Grid(nr, nphi, nz, 1.3, lz=5.0, policy=policy)
    s = _rand_spec(g, 7)
    back = O.forward(g, O.backward(g, s))
    assert O.spec_rel_err(g, back, s) < 1e-13


def test_backward_is_direct_sum():
    # Brute-force evaluation of Eq. (2) on a tiny grid, term by term.
    g = O.Grid(5, 6, 4, 0.8, lz=3.0, policy="linear")
    s = _rand_spec(g, 3)
    phys = O.backward(g, s)
    brute = np.zeros_like(phys)
    for l in range(g.nz):
        for j in range(g.nphi):
            for i in range(g.nr):
                acc = 0.0
                for m in range(-(g.M - 1), g.M):
                    am = abs(m)
                    for kk in range(g.K):
                        k = g.kz[kk]
                        for n in range(am, g.nc):
                            # shat_{n,-m,-k} = conj(shat_{n,m,k})
                            if m >= 0:
                                c = s[m][kk, n - m]
                            else:
                                kneg = int(np.where(g.kz == -k)[0][0])
                                c = np.conj(s[am][kneg, n - am])
                            if m == 0 and kk != 0:
                                pass
                            pn = (math.exp(O.ln_norm(n, am)) * (-1) ** am
                                  * sp.lpmv(am, n, g.x[i]))
                            acc += c * pn * np.exp(1j * (m * g.phi[j] + g.kappa[kk] * g.zz[l]))
                brute[l, j, i] = acc.real
    assert np.max(np.abs(phys - brute)) < 1e-12 * np.max(np.abs(brute))


def test_fourier_step_matches_numpy_fft():
    # Build each azimuthal band with numpy.fft from band-limited random Fourier
    # coefficients and give band m the radial profile Pbar_m^m; the forward
    # transform must return those coefficients in its n = m slot.
    g = O.Grid(8, 16, 8, 1.0, lz=2 * math.pi, policy="twothirds")
    rng = np.random.default_rng(5)
    phys = np.zeros((g.nz, g.nphi, g.nr))
    want = {}
    for m in range(g.M):
        C = np.zeros((g.nz, g.nphi), dtype=np.complex128)
        for kk in range(g.K):
            c = complex(rng.standard_normal(), rng.standard_normal())
            if m == 0 and g.kz[kk] == 0:
                c = c.real
            if m == 0 and g.kz[kk] < 0:
                continue
            want[(m, kk)] = c
            C[g.kz[kk] % g.nz, m] = c
            C[(-g.kz[kk]) % g.nz, (-m) % g.nphi] = np.conj(c)
        band = np.fft.ifft2(C).real * (g.nz * g.nphi)
        phys += band[:, :, None] * g.P[m][0][None, None, :]
    spec = O.forward(g, phys)
    for (m, kk), c in want.items():
        assert abs(spec[m][kk, 0] - c) < 1e-13
        if m == 0 and g.kz[kk] > 0:
            kneg = int(np.where(g.kz == -g.kz[kk])[0][0])
            assert abs(spec[0][kneg, 0] - np.conj(c)) < 1e-13
        assert np.all(np.abs(spec[m][kk, 1:]) < 1e-13)


def test_azimuthal_purity():
    # Sec. 5.1: for a cos(2 phi) field the odd harmonics vanish and the azimuthal
    # mean stays at round-off (the paper reports at most 8.5e-17).  The oracle's
    # naive DFT sums in matrix order, so its odd harmonics sit at round-off
    # rather than at an exact zero (an FFT's first butterfly makes them exact).
    for nr in (24, 48, 96):
        g = O.Grid(nr, 16, 1, 1.0)
        r, phi, z = g.nodes3()
        s = O.forward(g, W.heat_mode(r, phi, z, 0.0))
        scale = np.max(np.abs(s[2]))
        for m in range(1, g.M, 2):
            assert np.max(np.abs(s[m])) < 1e-15 * scale
        assert np.max(np.abs(s[0])) < 1e-16
        assert scale > 0.1


def test_representation_errors_match_paper(golden_dir):
    gold = json.load(open(os.path.join(golden_dir, "representation_errors.json")))
    for row in gold["s_B"]:
        g = O.Grid(row["nr"], 8, 1, row["ell"])
        r, phi, z = g.nodes3()
        f = W.field_sB(r, phi, z)
        err = O.weighted_l2(g, O.backward(g, O.forward(g, f)) - f, f)
        # two significant digits as printed
        assert float("%.1e" % err) == row["err"], (row, err)
    for row in gold["s_A"]:
        g = O.Grid(row["nr"], 8, 1, row["ell"])
        r, phi, z = g.nodes3()
        f = W.field_sA(r, phi, z)
        err = O.weighted_l2(g, O.backward(g, O.forward(g, f)) - f, f)
        assert err <= row["err_at_most"]


def test_flat_layout_roundtrip():
    g = O.Grid(10, 8, 6, 1.0, policy="twothirds")
    flat = W.random_spectral(g.nc, g.M, g.Kz, seed=1)
    assert np.array_equal(O.to_flat(g, O.from_flat(g, flat)), flat)
    # offset(m) = K * sum_{m' < m} (Nc - m')
    s = O.from_flat(g, flat)
    off = 0
    for m in range(g.M):
        assert np.array_equal(flat[off:off + g.K * (g.nc - m)], s[m].reshape(-1))
        off += g.K * (g.nc - m)
