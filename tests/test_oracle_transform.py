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


# --- Nyquist-keeping chop (|m| <= Nphi/2, |k| <= Nz/2): the aliased pair is split
# --- in equal halves in the forward direction and summed in the backward one.

def test_nyquist_chop_sizes():
    g = O.Grid(12, 8, 6, 1.0, policy="nyquist")
    assert (g.M, g.Kz, g.K) == (5, 4, 7)
    assert sorted(g.kz.tolist()) == [-3, -2, -1, 0, 1, 2, 3]
    g1 = O.Grid(12, 8, 1, 1.0, policy="nyquist")
    assert (g1.M, g1.Kz, g1.K) == (5, 1, 1)


@pytest.mark.parametrize("nphi,nz", [(8, 6), (16, 4), (4, 2)])
def test_nyquist_cosines_split_in_halves(nphi, nz):
    # cos(A) = (e^{iA} + e^{-iA}) / 2: a pure Nyquist cosine times a basis function
    # must come back as 1/2 in each stored member of the pair (1/4 per row for the
    # product of the azimuthal and the axial Nyquist cosines), and nothing else.
    g = O.Grid(nphi + 2, nphi, nz, 1.2, lz=3.0, policy="nyquist")
    r, phi, z = g.nodes3()
    mq, kq = nphi // 2, nz // 2
    prof_m = g.P[mq][0][None, None, :]       # Pbar_{mq}^{mq}(x_i), discrete-orthonormal
    prof_0 = g.P[0][0][None, None, :]
    cz = np.cos(2.0 * math.pi * kq * z / g.lz)
    cases = [
        (np.cos(mq * phi) * prof_m + 0 * z, mq, {0: 0.5}),
        (cz * prof_0 + 0 * phi, 0, {kq: 0.5, -kq: 0.5}),
        (np.cos(mq * phi) * cz * prof_m, mq, {kq: 0.25, -kq: 0.25}),
    ]
    for phys, m, want in cases:
        s = O.forward(g, phys)
        for mm in range(g.M):
            for kk in range(g.K):
                exp0 = want.get(int(g.kz[kk]), 0.0) if mm == m else 0.0
                assert abs(s[mm][kk, 0] - exp0) < 1e-14, (mm, kk)
                assert np.all(np.abs(s[mm][kk, 1:]) < 1e-14)


def test_nyquist_backward_closed_form():
    # one coefficient c at (n, m, k) = (Nphi/2, Nphi/2, 0): Eq. (2) with its
    # conjugate partner gives 2 Re(c e^{i (Nphi/2) phi_j}) = 2 Re(c) (-1)^j on the grid
    g = O.Grid(9, 8, 4, 0.9, lz=2.0, policy="nyquist")
    s = O.spec_zeros(g)
    c = 0.37 - 1.9j
    s[4][0, 0] = c
    phys = O.backward(g, s)
    r, phi, z = g.nodes3()
    want = 2.0 * c.real * np.cos(4 * phi) * g.P[4][0][None, None, :] + 0 * z
    assert np.max(np.abs(phys - want)) < 1e-14


def _nyquist_projection(g, s):
    """What forward(backward(s)) must return with the Nyquist kept: the m = Nphi/2
    block becomes its Hermitian part in k (its grid function is real), and the rows
    k = +-Nz/2 are replaced by their mean (they share one grid function)."""
    out = [b.copy() for b in s]
    idx = {int(k): i for i, k in enumerate(g.kz)}
    if g.nphi >= 2 and g.M - 1 == g.nphi // 2:
        b = out[g.M - 1]
        h = b.copy()
        for i, k in enumerate(g.kz):
            h[i] = 0.5 * (b[i] + np.conj(b[idx[-int(k)]]))
        out[g.M - 1] = h
    if g.nz > 1 and g.Kz - 1 == g.nz // 2:
        ip, im = idx[g.nz // 2], idx[-(g.nz // 2)]
        for b in out:
            avg = 0.5 * (b[ip] + b[im])
            b[ip] = avg
            b[im] = avg
    return out


@pytest.mark.parametrize("nr,nphi,nz", [(6, 4, 2), (9, 8, 4), (20, 16, 8), (33, 32, 16)])
def test_nyquist_roundtrip_is_the_pair_projection(nr, nphi, nz):
    g = O.Grid(nr, nphi, nz, 1.3, lz=5.0, policy="nyquist")
    s = _rand_spec(g, 11)
    back = O.forward(g, O.backward(g, s))
    want = _nyquist_projection(g, s)
    assert O.spec_rel_err(g, back, want) < 1e-13
    # and the projection is the identity on its own image
    again = O.forward(g, O.backward(g, want))
    assert O.spec_rel_err(g, again, want) < 1e-13


def test_nyquist_coefficient_matches_numpy_rfft():
    # the stored Nyquist coefficient of a random grid function equals numpy's real
    # DFT bin N/2 divided by 2N (Nz = 1, so only the azimuthal pair is involved)
    g = O.Grid(10, 16, 1, 1.0, policy="nyquist")
    rng = np.random.default_rng(4)
    a = rng.standard_normal(g.nphi)
    phys = a[None, :, None] * g.P[8][0][None, None, :]
    s = O.forward(g, phys)
    assert abs(s[8][0, 0] - np.fft.rfft(a)[8] / (2 * g.nphi)) < 1e-15
