"""Pins of the oracle's adaptive modal filter (Sec. 3.3; CPU only)."""

import math

import numpy as np
import pytest

import oracle as O
from oracle import filter as F
from paper_2609_18026_b300 import workloads as W


def _grid():
    return O.Grid(12, 16, 8, 1.0, lz=3.0, policy="twothirds")   # M = 6, Kz = 3, Nc = 12


def test_sigma_at_cutoff_and_edge():
    for eps in (0.0, 1.5, 36.0):
        assert F.sigma(2.0 / 3.0, eps, 2.0 / 3.0) == 1.0
        assert F.sigma(0.1, eps, 2.0 / 3.0) == 1.0
        assert abs(F.sigma(1.0, eps, 2.0 / 3.0) - math.exp(-eps)) <= 1e-16
        # half way between cutoff and edge: exp(-eps / 2^8)
        assert abs(F.sigma(5.0 / 6.0, eps, 2.0 / 3.0) - math.exp(-eps / 256.0)) <= 1e-15


def test_tail_fraction_brute_force():
    # every mode enumerated in plain loops: zeta = max(n/(Nc-1), m/(M-1), |k|/(Kz-1))
    g = _grid()
    spec = O.from_flat(g, W.random_spectral(g.nc, g.M, g.Kz, seed=3))
    zc = 0.55
    tail = tot = 0.0
    for m in range(g.M):
        for kk in range(g.K):
            k = abs(int(g.kz[kk]))
            for a, n in enumerate(range(m, g.nc)):
                z = max(n / (g.nc - 1), m / (g.M - 1), k / (g.Kz - 1))
                e = (1 if m == 0 else 2) * abs(spec[m][kk, a]) ** 2
                tot += e
                if z > zc:
                    tail += e
    assert abs(F.tail_fraction(g, spec, zc) - tail / tot) <= 1e-14


def test_field_below_target_passes_unchanged():
    # a spectrum decaying fast enough that the tail holds < tau of the energy:
    # eps stays 0 and every coefficient passes bit for bit
    g = _grid()
    spec = O.from_flat(g, W.random_spectral(g.nc, g.M, g.Kz, seed=4, scale_decay=1.5))
    for m in range(g.M):
        spec[m] *= np.exp(-2.5 * (m + np.abs(g.kz)))[:, None]
    assert F.tail_fraction(g, spec, F.DEFAULTS["zeta_c"]) < F.DEFAULTS["tau"]
    out, eps, f = F.apply(g, spec, 0.0)
    assert eps == 0.0
    for a, b in zip(out, spec):
        assert np.array_equal(a, b)


def test_relaxation_closed_form_and_damping():
    # white spectrum: the tail fraction is far above 2 tau, so eps* = eps_max and
    # eps_j = eps_max (1 - (1 - beta)^j); each mode is damped by sigma(zeta, eps_j)
    g = _grid()
    spec0 = O.from_flat(g, W.random_spectral(g.nc, g.M, g.Kz, seed=5))
    p = F.DEFAULTS
    spec, eps = spec0, 0.0
    for j in range(1, 5):
        f = F.tail_fraction(g, spec, p["zeta_c"])
        prev = spec
        spec, eps, f2 = F.apply(g, spec, eps)
        assert f2 == f
        if f >= 2 * p["tau"]:
            assert abs(eps - p["eps_max"] * (1 - (1 - p["relax"]) ** j)) <= 1e-12
        for m in range(g.M):
            for kk in range(g.K):
                z = F.zeta(g, m, kk)
                want = prev[m][kk] * np.where(z > p["zeta_c"], np.exp(-eps * np.clip(
                    (z - p["zeta_c"]) / (1 - p["zeta_c"]), 0, None) ** 8), 1.0)
                assert np.max(np.abs(spec[m][kk] - want)) <= 1e-15 * max(1.0, np.max(np.abs(want)))
    # the ramp: eps* is linear between tau and 2 tau
    assert F.update_eps(0.0, 1.5 * p["tau"], p["tau"], p["eps_max"], 1.0) == pytest.approx(0.5 * p["eps_max"])
    assert F.update_eps(10.0, 0.5 * p["tau"], p["tau"], p["eps_max"], 0.25) == pytest.approx(7.5)


def test_filter_between_steps_of_the_stepper():
    # the stepper applies the filter after every completed step (start and AB-CN)
    g = _grid()
    s0 = O.from_flat(g, W.random_spectral(g.nc, g.M, g.Kz, seed=6))
    filt = F.FieldFilter(g, 1)
    calls = []

    def post(s):
        calls.append(1)
        return filt(s)
    st = O.Stepper(g, 0.1, 1e-2, post=post)
    st.run_abcn(s0, 4)
    assert len(calls) == 4 and filt.eps[0] > 0.0
