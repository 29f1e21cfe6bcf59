"""Pins of the oracle's grid and basis against libraries and the paper (CPU only)."""

import math

import numpy as np
import pytest
import scipy.special as sp

import oracle as O


@pytest.mark.parametrize("n", [1, 2, 5, 24, 64, 128, 256])
def test_gauss_nodes_match_library(n):
    x, w = O.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.max(np.abs(x - xr)) < 2e-15
    # numpy's own end-node weights carry up to ~2e-11 relative error at n = 256
    # (checked against 40-digit values); the 40-digit test below is the tight pin
    assert np.max(np.abs(w - wr) / wr) < 5e-11
    assert abs(w.sum() - 2.0) < 1e-13


def test_gauss_weights_40_digits():
    import mpmath as mp
    mp.mp.dps = 40
    for n, idx in ((24, (0, 5, 11)), (64, (0, 1, 30)), (256, (0, 1, 128))):
        _check_mp(n, idx)


def _check_mp(n, idx):
    import mpmath as mp
    x, w = O.gauss_legendre(n)
    for i in idx:
        xi = mp.findroot(lambda t: mp.legendre(n, t), x[i])
        assert abs(float(xi) - x[i]) <= 2.3e-16
        dp = mp.diff(lambda t: mp.legendre(n, t), xi)
        we = 2 / ((1 - xi ** 2) * dp ** 2)
        assert abs(float((w[i] - we) / we)) < 5e-13


@pytest.mark.parametrize("n", [8, 33])
def test_gauss_rule_exact_for_monomials(n):
    x, w = O.gauss_legendre(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13


@pytest.mark.parametrize("n,ell", [(24, 1.0), (32, 4.0), (96, 0.5)])
def test_half_of_nodes_inside_ell(n, ell):
    # Sec. 3.1: ell places half of the Gauss-Legendre points within r < ell.
    g = O.Grid(n, 4, 1, ell)
    assert int(np.sum(g.r < ell)) == n // 2


def test_outermost_node_nr24():
    # Sec. 1 / grid figure: at Nr = 24 the outermost node lies 20-81 radii out for
    # the map scales shown; r_max / ell = 20.36.
    for ell in (1.0, 4.0):
        g = O.Grid(24, 16, 1, ell)
        assert abs(g.r[-1] / ell - 20.36) < 0.01


@pytest.mark.parametrize("nr,m", [(32, 0), (32, 5), (64, 31), (256, 128), (256, 200)])
def test_discrete_orthonormality(nr, m):
    x, w = O.gauss_legendre(nr)
    P = O.pbar_table(m + 1, nr, x)[m]
    G = (P * w[None, :]) @ P.T
    assert np.max(np.abs(G - np.eye(nr - m))) < 2e-13


@pytest.mark.parametrize("m", [0, 1, 3, 10, 40])
def test_pbar_matches_scipy_lpmv(m):
    nr = 64
    x, _ = O.gauss_legendre(nr)
    P = O.pbar_table(m + 1, nr, x)[m]
    for n in range(m, min(nr, m + 40)):
        ref = (-1) ** m * sp.lpmv(m, n, x) * math.exp(O.ln_norm(n, m))
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(P[n - m] - ref)) <= 1e-11 * max(scale, 1.0)


def test_pole_factor():
    # Sec. 3.1: Pbar_n^m carries (1-x^2)^{m/2}, so it is O(r^m) at the axis.
    x = np.array([-1.0 + 1e-8])
    for m in (1, 2, 3):
        P = O.pbar_table(m + 1, m + 6, x)[m]
        assert np.all(np.abs(P) < 1e-3 ** m * 10)
