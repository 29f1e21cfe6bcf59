"""Pins of the oracle's log proxy (Sec. 3.1, Eq. (6)) and of the enstrophy diagnostic
(CPU only)."""

import math

import numpy as np
import pytest
import scipy.special as sp
import sympy

import oracle as O
from oracle import logproxy as LP
from oracle.vortex import enstrophy

from vortex_states import q_vortex_state


def _lamb_oseen_psi_decay(r, gam, a, ell):
    """Decaying part psi - c Lambda (c = -gam / 4 pi) of the Lamb-Oseen stream
    function with lap_h psi = -omega, omega = gam / (pi a^2) exp(-r^2 / a^2):
    psi = -(gam / 4 pi) [E1(r^2/a^2) + ln(r^2/a^2)] + const, so that
    psi - c ln(r^2 + ell^2) = (gam / 4 pi) [ln(1 + ell^2 / r^2) - E1(r^2 / a^2)] + const,
    the constant chosen to make it vanish at infinity."""
    return gam / (4.0 * math.pi) * (np.log1p(ell * ell / (r * r)) - sp.exp1(r * r / (a * a)))


def _m0_block(g, f_nodes):
    """(0, 0) spectral block of an axisymmetric, z-independent field given at the nodes."""
    return O.forward(g, np.broadcast_to(f_nodes[None, None, :], (g.nz, g.nphi, g.nr)).copy())[0][0]


def test_image_is_the_laplacian_of_the_proxy():
    # backward of lam as the (0, 0) block is (1 - x)^2 / ell^2 at the nodes, which is
    # lap_h ln(r^2 + ell^2) = 4 ell^2 / (r^2 + ell^2)^2 (sympy)
    g = O.Grid(16, 4, 1, 1.7)
    s = O.spec_zeros(g)
    s[0][0] = LP.image(g.nc, g.ell)
    got = O.backward(g, s)[0, 0]
    rr, ll = sympy.symbols("r ell", positive=True)
    lam = sympy.log(rr ** 2 + ll ** 2)
    lap = sympy.simplify(sympy.diff(rr * sympy.diff(lam, rr), rr) / rr)
    want = sympy.lambdify((rr, ll), lap, "numpy")(g.r, g.ell)
    assert np.max(np.abs(got - want)) < 1e-14 * np.max(np.abs(want))
    assert np.max(np.abs(want - (1 - g.x) ** 2 / g.ell ** 2)) < 1e-14


@pytest.mark.parametrize("nr,ell,a", [(64, 1.5, 0.8), (96, 3.0, 1.0)])
def test_lamb_oseen_inversions(nr, ell, a):
    gam = 2.0 * math.pi
    g = O.Grid(nr, 4, 1, ell)
    D0 = O.del2h_closed(0, g.nc, g.ell)
    lam = LP.image(g.nc, g.ell)
    omega = gam / (math.pi * a * a) * np.exp(-g.r ** 2 / (a * a))
    f = _m0_block(g, -omega)                             # lap_h psi = -omega
    want = _m0_block(g, _lamb_oseen_psi_decay(g.r, gam, a, ell))
    # solve for c: the amplitude of the far field, and the basis part up to P_0^0
    s1, c1 = LP.solve_for_c(D0, lam, f)
    assert abs(c1 - (-gam / (4.0 * math.pi))) < 1e-10
    assert s1[0] == 0.0
    assert np.max(np.abs(s1[1:] - want[1:])) < 1e-9 * np.max(np.abs(want))
    # prescribed c: the decaying basis part itself
    s2 = LP.solve_prescribed(D0, lam, f, -gam / (4.0 * math.pi))
    assert np.max(np.abs(s2 - want)) < 1e-9 * np.max(np.abs(want))
    # the two variants differ only in the P_0^0 coefficient, up to the truncation of
    # f (the row the prescribed variant drops carries that residual)
    assert np.max(np.abs(s2[1:] - s1[1:])) < 1e-10 * np.max(np.abs(want))
    # the forward Laplacian of (s, c) gives the source back
    assert np.max(np.abs(LP.lap_apply(D0, lam, s1, c1) - f)) < 1e-10 * np.max(np.abs(f))
    # and with the wrong amplitude the decaying solve cannot reproduce the field
    s_bad = LP.solve_prescribed(D0, lam, f, 0.0)
    assert np.max(np.abs(s_bad - want)) > 1e-2 * np.max(np.abs(want))


def test_node_fields_against_sympy_and_legendre_forms():
    rr, ll, cp, cc = sympy.symbols("r ell c_psi c_chi", real=True)
    Lam = sympy.log(rr ** 2 + ll ** 2)
    lap = sympy.diff(rr * sympy.diff(Lam, rr), rr) / rr
    exact = {"v_phi": -cp * sympy.diff(Lam, rr),        # v = curl(psi e_z): v_phi = -d psi / dr
             "w_z": -cp * lap,                          # w_z = -lap_h psi
             "v_z": -cc * lap,                          # v_z = -lap_h chi
             "w_phi": cc * sympy.diff(lap, rr)}         # w_phi = d(lap chi) / dr
    g = O.Grid(24, 4, 1, 2.3)
    got = LP.node_fields(g.r, g.ell, 0.7, -1.3)
    for k, e in exact.items():
        v = sympy.lambdify((rr, ll, cp, cc), e, "numpy")(g.r, g.ell, 0.7, -1.3)
        assert np.max(np.abs(got[k] - v)) < 1e-13 * np.max(np.abs(v)), k
    # the Legendre forms of the r-weighted fields in x (what the CUDA path adds to
    # the (0, 0) blocks): r v_phi = -c_psi (1 + x), w_z = -c_psi (1 - x)^2 / ell^2,
    # v_z = -c_chi (1 - x)^2 / ell^2, r w_phi = -2 c_chi (1 - x)(1 - x^2) / ell^2
    x, e2 = g.x, g.ell ** 2
    assert np.allclose(g.r * got["v_phi"], -0.7 * (1 + x), rtol=0, atol=1e-14)
    assert np.allclose(got["w_z"], -0.7 * (1 - x) ** 2 / e2, rtol=0, atol=1e-14)
    assert np.allclose(got["v_z"], 1.3 * (1 - x) ** 2 / e2, rtol=0, atol=1e-14)
    assert np.allclose(g.r * got["w_phi"], 2.6 * (1 - x) * (1 - x * x) / e2, rtol=0, atol=1e-14)


@pytest.mark.parametrize("p", [4, 6, 8])
def test_hyperviscous_source_against_sympy(p):
    # L Lambda with nu = 0, nu_h = 1: -(-lap_h)^{p/2} Lambda = -(-1)^{p/2} lap_h^{p/2 - 1} [lap_h Lambda],
    # a polynomial of degree p in x, which the quadrature transform represents exactly
    g = O.Grid(32, 4, 1, 1.4)
    D0 = O.del2h_closed(0, g.nc, g.ell)
    src = LP.source(D0, LP.image(g.nc, g.ell), 0.0, 1.0, p)
    rr, ll = sympy.symbols("r ell", positive=True)
    f = sympy.log(rr ** 2 + ll ** 2)
    for _ in range(p // 2):
        f = sympy.simplify(sympy.diff(rr * sympy.diff(f, rr), rr) / rr)
    vals = -(-1.0) ** (p // 2) * sympy.lambdify((rr, ll), f, "numpy")(g.r, g.ell)
    want = _m0_block(g, vals)
    assert np.max(np.abs(src - want)) < 1e-11 * np.max(np.abs(want))
    assert np.all(src[p + 1:] == 0.0)


def test_diffusing_lamb_oseen_with_the_proxy_source():
    # omega(r, t) = gam / (pi a_t^2) exp(-r^2 / a_t^2), a_t^2 = a^2 + 4 nu t; the
    # amplitude c = -gam / (4 pi) stays fixed and the basis part follows the closed
    # form once the constant forcing c L Lambda is applied in the (0, 0) block
    gam, a, ell, nu, dt, nsteps = 2.0 * math.pi, 0.7, 1.5, 0.05, 2e-3, 250
    g = O.Grid(64, 4, 1, ell)
    c = -gam / (4.0 * math.pi)
    D0 = O.del2h_closed(0, g.nc, g.ell)
    lam = LP.image(g.nc, g.ell)
    s0 = O.spec_zeros(g)
    s0[0][0] = _m0_block(g, _lamb_oseen_psi_decay(g.r, gam, a, ell))
    src = c * LP.source(D0, lam, nu)

    def with_source(s):
        out = O.spec_zeros(g)
        out[0][0] = src.astype(np.complex128)
        return out

    def without(s):
        return O.spec_zeros(g)
    t = nsteps * dt
    want = _m0_block(g, _lamb_oseen_psi_decay(g.r, gam, math.sqrt(a * a + 4 * nu * t), ell))
    got, _ = O.Stepper(g, nu, dt, nonlinear=with_source).run_abcn(s0, nsteps)
    bad, _ = O.Stepper(g, nu, dt, nonlinear=without).run_abcn(s0, nsteps)
    err = np.max(np.abs(got[0][0] - want)) / np.max(np.abs(want))
    err_bad = np.max(np.abs(bad[0][0] - want)) / np.max(np.abs(want))
    assert err < 1e-6, err
    assert err_bad > 1e-2, err_bad


def _q_vortex_state(g, centres, q=1.0):
    return q_vortex_state(g, centres, q)


def test_shifted_q_vortex_is_steady():
    # a columnar vortex with an axial jet is a steady Euler flow wherever it sits, so
    # P[v x omega] vanishes (to the truncation of the fields); the flow has net
    # circulation 2 pi and net axial flux pi, carried by c_psi = -1/2, c_chi = -1/4
    g = O.Grid(56, 32, 1, 1.5)
    psi, chi, cp, cc, ops = _q_vortex_state(g, [(0.6, 0.0)])
    assert abs(cp + 0.5) < 1e-9 and abs(cc + 0.25) < 1e-9
    pN, cN = ops.nonlinear(psi, chi, 0.0, "plain", 0.0, cp, cc)
    pB, cB = ops.nonlinear(psi, chi, 0.0, "plain", 0.0, 0.0, 0.0)    # proxies dropped
    with_lp = O.spec_norm(g, pN) + O.spec_norm(g, cN)
    without = O.spec_norm(g, pB) + O.spec_norm(g, cB)
    assert with_lp < 1e-6 * without, (with_lp, without)
    # an axial background U_z adds U_z e_z x omega = -U_z w_phi e_r + U_z w_r e_phi,
    # whose curl is the advection -U_z d/dz: zero for a columnar flow
    pU, cU = ops.nonlinear(psi, chi, 0.0, "plain", -0.5, cp, cc)
    assert O.spec_norm(g, pU) + O.spec_norm(g, cU) < 1e-6 * without


def test_enstrophy_of_the_co_rotating_q_vortex_pair():
    # omega = (grad v_z x e_z, w_z) with w_z = 2 e^{-rho^2}, v_z = e^{-rho^2} per
    # vortex: int |omega|^2 dA = 3 pi per vortex and 2 (2 pi - 7 pi) e^{-b^2/2} for
    # the cross terms, b = 4; Z = (1/2) Lz int |omega|^2 dA
    g = O.Grid(64, 64, 1, 4.0, lz=2.0 * math.pi)
    psi, chi, cp, cc, ops = _q_vortex_state(g, [(2.0, 0.0), (-2.0, 0.0)])
    assert abs(cp + 1.0) < 1e-8 and abs(cc + 0.5) < 1e-8
    Z, wmax = enstrophy(g, ops, psi, chi, cp, cc)
    want = 0.5 * g.lz * (6.0 * math.pi - 10.0 * math.pi * math.exp(-8.0))
    assert abs(Z - want) < 1e-6 * want, (Z, want)
    Zb, _ = enstrophy(g, ops, psi, chi, 0.0, 0.0)
    assert abs(Zb - want) > 1e-2 * want
    # the peak |omega| sits near each centre, where w_z = 2 (1 + e^{-16}) and
    # w_phi = 0; the nodes miss the centre by less than a grid spacing
    assert 1.9 < wmax <= 2.0 + 1e-6
