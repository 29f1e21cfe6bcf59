"""Pins of the oracle's operators and integrators (CPU only)."""

import json
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle.operators import del2h_unnormalised, logproxy_image
from paper_2609_18026_b300 import workloads as W


@pytest.mark.parametrize("nc,m,ell", [(16, 0, 1.0), (32, 1, 2.0), (64, 3, 0.7),
                                      (64, 7, 4.0), (128, 40, 1.0), (256, 85, 1.0)])
def test_laplacian_two_constructions_agree(nc, m, ell):
    A = O.del2h_closed(m, nc, ell)
    B = O.del2h_quadrature(m, nc, ell)
    assert np.max(np.abs(A - B)) <= 1e-12 * np.max(np.abs(B))
    # pentadiagonal
    idx = np.arange(A.shape[0])
    assert np.all(A[np.abs(idx[:, None] - idx[None, :]) > 2] == 0.0)


def test_laplacian_hand_closed_form():
    # ell^2 lap P_1^0 = 4/3 P_0 - 16/5 P_1 + 8/3 P_2 - 4/5 P_3 (unnormalised basis),
    # derived by hand from Eq. (3): lap_h P_n = -n(n+1)(1-x)^2 ell^-2 P_n, with
    # (1-x)^2 x = x - 2x^2 + x^3 expanded in Legendre polynomials.
    D = del2h_unnormalised(0, 8, 1.0)
    col = D[:, 1]
    assert np.allclose(col[:4], [4 / 3, -16 / 5, 8 / 3, -4 / 5], rtol=0, atol=1e-15)
    assert np.all(col[4:] == 0.0)


def test_logproxy_image():
    # Eq. (6): (4/3 P0 - 2 P1 + 2/3 P2)/ell^2 == lap_h ln(r^2+ell^2) = (1-x)^2/ell^2
    x = np.linspace(-0.99, 0.99, 41)
    c = logproxy_image(2.0)
    val = c[0] + c[1] * x + c[2] * 0.5 * (3 * x * x - 1)
    assert np.max(np.abs(val - (1 - x) ** 2 / 4.0)) < 1e-15


def test_laplacian_spectral_accuracy_on_sB():
    # lap_h [r^2 e^{-r^2/2} cos 2phi] = (r^4 - 6 r^2) e^{-r^2/2} cos 2phi
    g = O.Grid(64, 8, 1, 2.0)
    r, phi, z = g.nodes3()
    s = O.forward(g, W.field_sB(r, phi, z))
    lap = [O.del2h_closed(m, g.nc, g.ell) @ s[m][0] for m in range(g.M)]
    exact = (r ** 4 - 6 * r ** 2) * np.exp(-r ** 2 / 2) * np.cos(2 * phi) + 0 * z
    ref = O.forward(g, exact)
    for m in range(g.M):
        assert np.max(np.abs(lap[m] - ref[m][0])) < 1e-7


def test_rdr_spectral_accuracy_on_sB():
    # r d/dr [r^2 e^{-r^2/2}] = (2 r^2 - r^4) e^{-r^2/2}; tridiagonal
    g = O.Grid(64, 8, 1, 2.0)
    r, phi, z = g.nodes3()
    s = O.forward(g, W.field_sB(r, phi, z))
    R = O.rdr_matrix(2, g.nc)
    idx = np.arange(R.shape[0])
    assert np.all(R[np.abs(idx[:, None] - idx[None, :]) > 1] == 0.0)
    got = R @ s[2][0]
    exact = (2 * r ** 2 - r ** 4) * np.exp(-r ** 2 / 2) * np.cos(2 * phi) + 0 * z
    ref = O.forward(g, exact)[2][0]
    assert np.max(np.abs(got - ref)) < 1e-7


def test_rdr_of_basis_function_by_quadrature():
    # Independent check: project (1-x^2) d/dx Pbar_n^m (finite differences of the
    # recurrence at shifted nodes would be noisy; use the analytic derivative of
    # the unnormalised Ferrers function from scipy) onto the basis.
    import scipy.special as sp
    m, nc = 3, 20
    xq, wq = O.gauss_legendre(nc + 4)
    P = O.pbar_table(m + 1, nc + 2, xq)[m]
    R = O.rdr_matrix(m, nc)
    for n in range(m, nc - 1):
        # d/dx of Ferrers P_n^m via lpmv derivative identity
        # (1-x^2) P' = (n+m) P_{n-1} - n x P_n   (no phase)
        pn = (-1) ** m * sp.lpmv(m, n, xq)
        pn1 = (-1) ** m * sp.lpmv(m, n - 1, xq) if n - 1 >= m else 0.0 * xq
        f = ((n + m) * pn1 - n * xq * pn) * math.exp(O.ln_norm(n, m))
        proj = (P * wq[None, :]) @ f
        col = R[:, n - m]
        assert np.max(np.abs(proj[: nc - m] - col)) < 1e-12 * max(1.0, np.max(np.abs(col)))


def _oseen_run(scheme, dt):
    g = O.Grid(96, 1, 1, 1.0, M=1)
    r, phi, z = g.nodes3()
    st = O.Stepper(g, 0.1, dt)
    s0 = O.forward(g, W.oseen(r, phi, z, 0.0))
    n = int(round(10.0 / dt))
    s = st.run_abcn(s0, n)[0] if scheme == "abcn" else st.run_febe(s0, n)
    u = O.backward(g, s)
    ex = W.oseen(r, phi, z, 10.0)
    return O.weighted_l2(g, u - ex, ex), O.circulation(g, u), O.second_moment(g, u)


def test_oseen_table2_every_digit(golden_dir):
    gold = json.load(open(os.path.join(golden_dir, "oseen_table2.json")))
    for row in gold["rows"]:
        err, gam, m2 = _oseen_run(row["scheme"], row["dt"])
        assert float("%.3e" % err) == row["rel_l2w"] or abs(err / row["rel_l2w"] - 1) < 1e-4, (row, err)
        assert "%.7f" % gam == row["gamma"], (row, gam)
        assert "%.4f" % m2 == row["m2"], (row, m2)


def test_oseen_richardson_start_matters():
    # Without the Richardson start (AB-CN from A^{-1} = A^0 = 0 with a plain CN
    # first step) the Gamma digits differ from Table 2: the start-up is pinned.
    g = O.Grid(96, 1, 1, 1.0, M=1)
    r, phi, z = g.nodes3()
    st = O.Stepper(g, 0.1, 1.0)
    s0 = O.forward(g, W.oseen(r, phi, z, 0.0))
    zero = [np.zeros_like(b) for b in s0]
    s, _ = st.run_abcn_from(s0, zero, 10)
    u = O.backward(g, s)
    assert "%.7f" % O.circulation(g, u) != "0.9999945"


@pytest.mark.slow
def test_fkpp_linearised_solution(golden_dir):
    gold = json.load(open(os.path.join(golden_dir, "fkpp_linear.json")))
    g = O.Grid(96, 1, 1, 4.0, M=1)
    r, phi, z = g.nodes3()
    for row in gold["rows"]:
        st = O.Stepper(g, 1.0, row["dt"], nonlinear=O.fkpp_nonlinear(g, 0.25))
        s, _ = st.run_abcn(O.forward(g, W.kpp_linear(r, phi, z, 0.0)), int(round(20.0 / row["dt"])))
        u = O.backward(g, s)
        ex = W.kpp_linear(r, phi, z, 20.0)
        err = O.weighted_l2(g, u - ex, ex)
        fmt = "%%.%de" % (row["digits"] - 1)
        assert float(fmt % err) == row["rel_l2w"], (row, err)


def test_heat_mode_design_orders():
    # Eq. (15), m = 2: FE-BE first order, AB-CN second order in dt (Sec. 5.1).
    # Nr = 96 keeps the spatial error (2.7e-7 in the paper) below the temporal one.
    g = O.Grid(96, 8, 1, 1.0)
    r, phi, z = g.nodes3()
    s0 = O.forward(g, W.heat_mode(r, phi, z, 0.0))
    ex = W.heat_mode(r, phi, z, 1.0)
    errs = {"febe": [], "abcn": []}
    for dt in (0.05, 0.025, 0.0125):
        st = O.Stepper(g, 0.1, dt)
        n = int(round(1.0 / dt))
        for sch in errs:
            s = st.run_abcn(s0, n)[0] if sch == "abcn" else st.run_febe(s0, n)
            errs[sch].append(O.weighted_l2(g, O.backward(g, s) - ex, ex))
    p_fb = math.log2(errs["febe"][1] / errs["febe"][2])
    p_ab0 = math.log2(errs["abcn"][0] / errs["abcn"][1])
    p_ab = math.log2(errs["abcn"][1] / errs["abcn"][2])
    assert 0.95 < p_fb < 1.05, errs
    # approaches 2 from below as in Table 2 (1.898, 1.938)
    assert 1.85 < p_ab < 2.05 and p_ab > p_ab0, errs


def test_polar_diffusion_closed_form():
    # Pole-regular variant of the 2-D polar diffusion seed: exact solution
    # B^-1 e^{-r^2/B} + 0.5 r^2 B^-3 e^{-r^2/B} cos 2 phi, B = 1 + 4 nu t
    # (Eq. (15) with sigma0^2 = 1/2).  nu = 1e-2, 100 AB-CN steps of 1e-3 as in the
    # 2-D polar workload, at Nr = 64 so that the Gaussian's representation error
    # (5e-6 at Nr = 32, ell = 1) is below the bound checked.
    nu, dt, n = 1e-2, 1e-3, 100
    g = O.Grid(64, 32, 1, 1.0)
    r, phi, z = g.nodes3()
    st = O.Stepper(g, nu, dt)
    s, _ = st.run_abcn(O.forward(g, W.gaussian_polar_reg(r, phi, z)), n)
    t = n * dt
    B = 1 + 4 * nu * t
    ex = np.exp(-r ** 2 / B) / B + 0.5 * r ** 2 * np.exp(-r ** 2 / B) / B ** 3 * np.cos(2 * phi) + 0 * z
    assert O.weighted_l2(g, O.backward(g, s) - ex, ex) < 1e-7


def test_norm_ratio_matches_log_form():
    # The exact ratio agrees with the paper's exp(ln N_j - ln N_n) form to the
    # accuracy of the rounded logs.
    from oracle.operators import norm_ratio
    for m in (0, 3, 50):
        for n in range(m, m + 120, 7):
            for j in (n - 2, n - 1, n + 1, n + 2):
                if j < m:
                    continue
                lg = math.exp(O.ln_norm(j, m) - O.ln_norm(n, m))
                assert abs(norm_ratio(j, n, m) / lg - 1) < 1e-12


def _iterated_laplacian(j, kappa):
    """(d^2/dr^2 + 1/r d/dr - 4/r^2 - kappa^2)^j of r^2 e^{-r^2/2} (the m = 2
    profile of s_B), in closed form by sympy, as a numpy function of r."""
    import sympy as sp
    rs = sp.symbols("r", positive=True)
    f = rs ** 2 * sp.exp(-rs ** 2 / 2)
    for _ in range(j):
        f = sp.expand(sp.diff(f, rs, 2) + sp.diff(f, rs) / rs - 4 * f / rs ** 2 - sp.Float(kappa) ** 2 * f)
    return sp.lambdify(rs, f, "numpy")


@pytest.mark.parametrize("p,tol", [(4, 1e-9), (6, 1e-7), (8, 1e-5)])
@pytest.mark.parametrize("kappa", [0.0, 0.7])
def test_hyperviscous_power_against_iterated_laplacian(p, tol, kappa):
    # Eq. (11) with nu = 0, nu_h = 1: L s = -(-lap)^{p/2} s = -(-1)^{p/2} lap^{p/2} s,
    # lap = D_m - kappa^2 on the harmonic (m = 2, kappa) of s_B (Eq. (13)).  The
    # expected coefficients come from the iterated analytic Laplacian of
    # r^2 e^{-r^2/2}; rows below Nc - m - p are untouched by the truncation.  A
    # wrong exponent (p instead of p/2) or sign fails by O(1).
    g = O.Grid(64, 8, 1, 2.0)
    r, phi, z = g.nodes3()
    s = O.forward(g, W.field_sB(r, phi, z))[2][0]
    L = O.linear_operator(2, kappa, g.nc, g.ell, 0.0, 1.0, p)
    f = _iterated_laplacian(p // 2, kappa)
    exact = -(-1) ** (p // 2) * f(r) * np.cos(2 * phi) + 0 * z
    ref = O.forward(g, exact)[2][0]
    k = g.nc - 2 - p
    assert np.max(np.abs((L @ s)[:k] - ref[:k])) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("m,nc,kappa", [(0, 24, 0.0), (3, 40, 1.3), (7, 33, 0.4)])
@pytest.mark.parametrize("p", [4, 6, 8])
def test_dissipation_truncate_then_compose(m, nc, kappa, p):
    # Eq. (11) read as powers of the truncated (Nc - m) x (Nc - m) Laplacian
    # ("shifting and composing", Sec. 3.1): built here from the independent
    # quadrature construction of D_m (Eq. (3)) and a library matrix power, with
    # nu and nu_h both nonzero.  Compose-then-truncate would differ in the last p
    # rows; a wrong exponent or sign everywhere.
    ell, nu, nu_h = 1.7, 0.3, 2e-3
    D = O.del2h_quadrature(m, nc, ell)
    lap = D - kappa * kappa * np.eye(nc - m)
    ref = nu * lap - nu_h * np.linalg.matrix_power(-lap, p // 2)
    L = O.linear_operator(m, kappa, nc, ell, nu, nu_h, p)
    assert np.max(np.abs(L - ref)) <= 1e-10 * np.max(np.abs(ref))
    # the reading is visible: the composed power of a larger matrix, truncated
    # afterwards, differs in the last rows
    Dbig = O.del2h_quadrature(m, nc + p, ell)
    lbig = Dbig - kappa * kappa * np.eye(nc + p - m)
    ctt = np.linalg.matrix_power(-lbig, p // 2)[: nc - m, : nc - m]
    assert np.max(np.abs(ctt[-1] - np.linalg.matrix_power(-lap, p // 2)[-1])) > 1e-3 * np.max(np.abs(ctt))


def _pbar_lib(n, m, x):
    """Normalised associated Legendre function from scipy's Ferrers function
    (which carries the (-1)^m Condon-Shortley phase) and the exact norm of Eq. (7)."""
    import scipy.special as sp
    return (-1) ** m * sp.lpmv(m, n, x) * math.sqrt((2 * n + 1) * math.factorial(n - m)
                                                      / (2.0 * math.factorial(n + m)))


@pytest.mark.parametrize("m1,k1,gamma", [(2, 1, 1.0), (3, 2, 0.25)])
def test_fkpp_product_and_two_thirds_mask(m1, k1, gamma):
    # Eq. (17): A = gamma u (1 - u) at the nodes, forward transform, two-thirds
    # mask (Sec. 3.3).  u = a Pbar_5^{m1}(x) cos(m1 phi) cos(kappa_{k1} z)
    # + b Pbar_3^0(x) is band-limited so that u^2 is alias-free on the grid
    # (2 m1 < Nphi / 2, 2 k1 <= Nz / 2, radial degrees within the Gauss rule);
    # the retained modes of gamma u (1 - u) are then exact.  Expected values:
    # quadrature of the analytic product on an independent 80-point Gauss rule
    # (numpy leggauss), basis from scipy's Ferrers functions, exact DFTs on 32
    # points per periodic direction (numpy.fft).  (m1, k1) = (2, 1) keeps the
    # m = 4, |k| = 2 products (M = 6, Kz = 3); (3, 2) masks them (2 m1 = 6 >= M,
    # 2 k1 = 4 >= Kz).  A missing -gamma u^2 term, a wrong sign or an aliased
    # product fails.
    nr, nphi, nz, ell, lz = 16, 16, 8, 1.3, 5.0
    a, b, n1, n2 = 0.6, 0.8, 5, 3
    g = O.Grid(nr, nphi, nz, ell, lz=lz, policy="twothirds")
    assert (g.M, g.Kz) == (6, 3)
    spec = O.spec_zeros(g)
    kidx = {int(k): i for i, k in enumerate(g.kz)}
    spec[0][0, n2] = b
    for sgn in (1, -1):
        spec[m1][kidx[sgn * k1], n1 - m1] = a / 4.0
    out = O.fkpp_nonlinear(g, gamma)(spec)

    xq, wq = np.polynomial.legendre.leggauss(80)
    nf = 32
    ph = 2 * math.pi * np.arange(nf) / nf
    zz = lz * np.arange(nf) / nf
    kap1 = 2 * math.pi * k1 / lz
    u = (a * _pbar_lib(n1, m1, xq)[:, None, None] * np.cos(m1 * ph)[None, :, None]
         * np.cos(kap1 * zz)[None, None, :] + b * _pbar_lib(n2, 0, xq)[:, None, None])
    F = gamma * u * (1.0 - u)
    Fh = np.fft.fft(np.fft.fft(F, axis=1), axis=2) / (nf * nf)   # [x][m][k]
    for m in range(g.M):
        for kk in range(g.K):
            k = int(g.kz[kk])
            prof = Fh[:, m, k % nf]
            for n in range(m, g.nc):
                exp_c = np.sum(wq * _pbar_lib(n, m, xq) * prof)
                assert abs(out[m][kk, n - m] - exp_c) < 1e-13, (m, k, n, out[m][kk, n - m], exp_c)


def test_fkpp_uniform_state_follows_the_logistic_closed_form():
    # Eq. (17) with a spatially uniform state: the Laplacian annihilates the n = 0
    # mode, so the whole nonlinear evolution reduces to u' = gamma u (1 - u), whose
    # solution is u0 e^{gamma t} / (1 - u0 + u0 e^{gamma t}).  This pins the product,
    # both transforms and the Richardson-started AB-CN stepping of the oracle beyond
    # the linear regime: the state stays uniform, and its error against the closed
    # form is second order in dt.
    g = O.Grid(12, 4, 4, 1.0, lz=3.0)
    r, phi, z = g.nodes3()
    u0, gamma, T = 0.1, 1.0, 3.0
    exact = u0 * math.exp(gamma * T) / (1.0 - u0 + u0 * math.exp(gamma * T))
    errs = []
    for dt in (0.05, 0.025):
        st = O.Stepper(g, 0.5, dt, nonlinear=O.fkpp_nonlinear(g, gamma))
        s0 = O.forward(g, np.full(np.broadcast(r, phi, z).shape, u0))
        s, _ = st.run_abcn(s0, int(round(T / dt)))
        u = O.backward(g, s)
        assert np.ptp(u) <= 1e-12
        errs.append(abs(float(np.mean(u)) - exact))
    assert errs[0] <= 2e-3 * exact
    assert 3.2 <= errs[0] / errs[1] <= 4.8, errs
