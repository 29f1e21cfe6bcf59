"""Pins of the oracle's toroidal-poloidal vortex term (CPU only)."""

import math

import numpy as np
import pytest

import oracle as O
from paper_2609_18026_b300 import workloads as W


def _grid():
    return O.Grid(40, 8, 8, 1.0, lz=2 * math.pi, policy="linear")


def _nodes(g):
    return g.nodes3()


@pytest.mark.parametrize("form", ["plain", "banded"])
def test_gradient_field_projects_to_zero(form):
    # N = grad g with g = f(r) cos 2phi cos z, f = r^2/(r^2+a^2)^3 (rational, so
    # analytic in the mapped coordinate and resolved to round-off as s_A of
    # Sec. 5.1): curl N = 0 and the gradient part is removed, so P(N) = (0, 0)
    # (Sec. 3.2: the projection removes any gradient contribution).
    g = _grid()
    ops = O.VortexOps(g)
    r, phi, z = _nodes(g)
    kap = 2 * math.pi / g.lz
    a2 = 1.3 ** 2
    q = r ** 2 + a2
    f = r ** 2 / q ** 3
    fp = 2 * r / q ** 3 - 6 * r ** 3 / q ** 4
    A = -2 * f * np.sin(2 * phi) * np.cos(kap * z)          # r N_phi = d_phi g
    Bf = r * fp * np.cos(2 * phi) * np.cos(kap * z)         # r N_r = r d_r g
    Nz = -kap * f * np.cos(2 * phi) * np.sin(kap * z)       # N_z = d_z g
    if form == "plain":
        psiN, chiN = ops.project_plain(O.forward(g, A), O.forward(g, Bf), O.forward(g, Nz))
    else:
        psiN, chiN = ops.project_banded(O.forward(g, A), O.forward(g, Bf), O.forward(g, r ** 2 * Nz))
    scale = O.spec_norm(g, O.forward(g, f * np.cos(2 * phi) * np.cos(kap * z)))
    assert O.spec_norm(g, psiN) < 1e-9 * scale
    assert O.spec_norm(g, chiN) < 1e-9 * scale


@pytest.mark.parametrize("form", ["plain", "banded"])
def test_solenoidal_field_projects_back(form):
    # V = curl(psi e_z) + curl curl(chi e_z) with rational decaying psi (m = 2)
    # and chi (m = 1): P(V) returns (psi, chi) (Eq. (8)-(9)).
    g = _grid()
    ops = O.VortexOps(g)
    r, phi, z = _nodes(g)
    kap = 2 * math.pi / g.lz
    q = r ** 2 + 1.3 ** 2
    psi = O.forward(g, r ** 2 / q ** 2 * np.cos(2 * phi) * np.cos(kap * z))
    chi = O.forward(g, r / q ** 2 * np.cos(phi) * np.sin(kap * z))
    rvr, rvp, vz, _, _, _ = ops.fields(psi, chi)
    if form == "plain":
        pN, cN = ops.project_plain(rvp, rvr, vz)
    else:
        pN, cN = ops.project_banded(rvp, rvr, O.forward(g, r ** 2 * O.backward(g, vz)))
    assert O.spec_rel_err(g, pN, psi) < 1e-8
    assert O.spec_rel_err(g, cN, chi) < 1e-8


def test_vorticity_fields_match_analytic_curl():
    # psi = -(1 + r^2)^-2 (m = 0, k = 0): v_phi = -d_r psi = -4 r (1 + r^2)^-3 and
    # w_z = -lap_h psi = (16 r^2 - 8) (1 + r^2)^-4.
    g = O.Grid(48, 4, 1, 1.0)
    ops = O.VortexOps(g)
    r, phi, z = g.nodes3()
    q = 1 + r ** 2
    psi = O.forward(g, -q ** -2 + 0 * phi + 0 * z)
    chi = [np.zeros_like(b) for b in psi]
    rvr, rvp, vz, rwr, rwp, wz = (O.backward(g, f) for f in ops.fields(psi, chi))
    vphi = -4 * r / q ** 3 + 0 * phi + 0 * z
    assert np.max(np.abs(rvp - r * vphi)) < 1e-10
    assert np.max(np.abs(wz - (16 * r ** 2 - 8) / q ** 4)) < 1e-10
    assert np.max(np.abs(rvr)) < 1e-12 and np.max(np.abs(vz)) < 1e-12


@pytest.mark.parametrize("form", ["plain", "banded"])
def test_axisymmetric_vortex_has_no_projected_forcing(form):
    # A shielded axisymmetric vortex (psi = -e^{-r^2}, zero net circulation):
    # N = (v_phi w_z) e_r is a pure gradient, so P(N) = 0 (the steady Euler
    # balance of a columnar vortex).
    g = O.Grid(48, 4, 4, 1.0, lz=4.0)
    ops = O.VortexOps(g)
    r, phi, z = g.nodes3()
    psi = O.forward(g, -np.exp(-r ** 2) + 0 * phi + 0 * z)
    chi = [np.zeros_like(b) for b in psi]
    pN, cN = ops.nonlinear(psi, chi, U0=0.0, form=form)
    assert O.spec_norm(g, pN) < 1e-9 * O.spec_norm(g, psi)
    assert O.spec_norm(g, cN) < 1e-9 * O.spec_norm(g, psi)


@pytest.mark.parametrize("form", ["plain", "banded"])
@pytest.mark.parametrize("U0", [1.0, -1.0])
def test_uniform_background_translates_axisymmetric_vortex(form, U0):
    # Moving frame (Sec. 5.3): a shielded axisymmetric vortex psi = -(1 + r^2)^-2
    # (rational, resolved to round-off; zero net circulation) in the background
    # U = U0 e_y.  v x omega is a gradient (previous test); U x omega =
    # U0 w_z e_x has (curl)_z = -U0 d(w_z)/dy, so psi_N = -lap_h^{-1} of it =
    # -U0 d(psi)/dy = -U0 psi'(r) sin(phi) = -4 U0 r (1 + r^2)^-3 sin(phi) in
    # closed form (pure translation of psi along y), and chi_N = 0 (N_z = 0,
    # k = 0).  A sin/cos swap or a sign error in U_r = U0 sin(phi),
    # U_phi = U0 cos(phi) moves this to cos(phi) or flips it.
    g = O.Grid(48, 8, 1, 1.0)
    ops = O.VortexOps(g)
    r, phi, z = g.nodes3()
    psi = O.forward(g, -(1.0 + r ** 2) ** -2.0 + 0 * phi + 0 * z)
    chi = [np.zeros_like(b) for b in psi]
    pN, cN = ops.nonlinear(psi, chi, U0=U0, form=form)
    exact = O.forward(g, -4.0 * U0 * r * (1.0 + r ** 2) ** -3.0 * np.sin(phi) + 0 * z)
    assert O.spec_rel_err(g, pN, exact) < 1e-8
    assert O.spec_norm(g, cN) < 1e-9 * O.spec_norm(g, exact)


def test_plain_and_banded_projection_converge_to_one_limit():
    # The two evaluations of P agree in exact arithmetic and differ on a
    # truncated expansion only by the truncation of the products.  For one
    # resolved input (Nc0 = 32 coefficients decaying like e^{-n}, zero-padded to
    # larger Nr) the plain - banded difference must fall as Nr grows, and both
    # forms must approach the finest plain result.  psi converges spectrally;
    # chi more slowly, through g = (lap - kappa^2)^{-1} div N ~ e^{-kappa r},
    # which is smooth but not analytic in the mapped coordinate at r = inf.
    nphi, nz = 16, 8
    g0 = O.Grid(32, nphi, nz, 1.0, lz=8.6, policy="twothirds")
    psi0 = O.from_flat(g0, W.random_spectral(g0.nc, g0.M, g0.Kz, seed=11, scale_decay=1.0))
    chi0 = O.from_flat(g0, W.random_spectral(g0.nc, g0.M, g0.Kz, seed=12, scale_decay=1.0))

    def pad(g, s):
        return [np.concatenate([s[m], np.zeros((g.K, g.nc - g0.nc), complex)], axis=1) for m in range(g.M)]

    def cut(s):
        return [s[m][:, :g0.nc - m] for m in range(g0.M)]

    out = {}
    for nr in (48, 96, 192):
        g = O.Grid(nr, nphi, nz, 1.0, lz=8.6, policy="twothirds")
        ops = O.VortexOps(g)
        for form in ("plain", "banded"):
            p, c = ops.nonlinear(pad(g, psi0), pad(g, chi0), 1.0, form)
            out[(nr, form)] = (cut(p), cut(c))

    def diff(a, b):
        return max(O.spec_rel_err(g0, a[0], b[0]), O.spec_rel_err(g0, a[1], b[1]))

    d = [diff(out[(nr, "banded")], out[(nr, "plain")]) for nr in (48, 96, 192)]
    # measured: 8.4e-6, 1.0e-7, 1.4e-9
    assert d[0] < 5e-5 and d[1] < 1e-6 and d[2] < 2e-8
    assert d[0] > 10 * d[1] > 100 * d[2]
    ref = out[(192, "plain")]
    for form in ("plain", "banded"):
        e48, e96 = diff(out[(48, form)], ref), diff(out[(96, form)], ref)
        assert e96 < 0.1 * e48 and e96 < 1e-6


def test_lap_h_inverse_decay_row():
    # D_m x = f then D_m x reproduces f (rows n >= 1 at m = 0); x decays at r -> inf
    g = O.Grid(32, 4, 1, 1.0)
    ops = O.VortexOps(g)
    r, phi, z = g.nodes3()
    q = 1 + r ** 2
    f = O.forward(g, (16 * r ** 2 - 8) / q ** 4 + 0 * phi + 0 * z)[0][0]
    x = ops.lap_h_inv(0, f)
    assert np.max(np.abs((ops.D[0] @ x)[1:] - f[1:])) < 1e-10
    assert abs(np.sum(x * O.vortex.pbar_at_one(0, g.nc))) < 1e-12
    exact = O.forward(g, q ** -2 + 0 * phi + 0 * z)[0][0]   # lap_h (1+r^2)^-2 = f, decays
    assert np.max(np.abs(x - exact)) < 1e-10


def test_jacobi_and_r2_laplacian_by_quadrature():
    # J = <Pbar_j, x Pbar_n> and Q = <Pbar_j, r^2 lap_h Pbar_n> = -n(n+1) <Pbar_j, (1-x^2) Pbar_n>
    # by Gauss quadrature (exact with Nc + 2 nodes); interior block (truncation
    # affects only the last rows of the composed Q)
    from oracle.vortex import jacobi_matrix
    for m, nc in ((0, 12), (3, 20)):
        xq, wq = O.gauss_legendre(nc + 4)
        P = O.pbar_table(m + 1, nc + 2, xq)[m]
        Jq = (P * (wq * xq)[None, :]) @ P.T
        J = jacobi_matrix(m, nc)
        assert np.max(np.abs(J - Jq[: nc - m, : nc - m])) < 1e-14
        n = np.arange(m, nc + 2, dtype=float)
        Qq = ((P * (wq * (1 - xq ** 2))[None, :]) @ P.T) * (-n * (n + 1))[None, :]
        ops = O.VortexOps(O.Grid(nc, 2 * (m + 1) + 2, 1, 1.0, M=m + 1, nr_c=nc))
        Q = ops.Q[m]
        k = nc - m - 2
        assert np.max(np.abs(Q[:k, :k] - Qq[:k, :k])) < 1e-11 * np.max(np.abs(Qq))


def test_axial_energy_closed_form():
    # psi = -(1 + r^2)^-2 (axisymmetric, k = 0): v_phi = 4 r (1 + r^2)^-3 and
    # E_0 = (1/2) Lz 2 pi int 16 r^3 (1 + r^2)^-6 dr = 16 pi Lz / 40 = 0.4 pi Lz;
    # adding a k = 1 poloidal perturbation puts energy in E_1 only (linear in the
    # perturbation's square), leaving E_0 unchanged to round-off
    from oracle.vortex import axial_energy
    g = O.Grid(48, 8, 8, 1.0, lz=5.0)
    ops = O.VortexOps(g)
    r, phi, z = g.nodes3()
    psi = O.forward(g, -(1.0 + r ** 2) ** -2.0 + 0 * phi + 0 * z)
    chi = [np.zeros_like(b) for b in psi]
    E = axial_energy(g, ops, psi, chi)
    assert abs(E[0] - 0.4 * math.pi * g.lz) <= 1e-10 * E[0]
    assert np.all(np.abs(E[1:]) <= 1e-20)
    kap = 2 * math.pi / g.lz
    chi1 = O.forward(g, 1e-3 * r ** 2 / (1 + r ** 2) ** 2 * np.cos(kap * z) + 0 * phi)
    E2 = axial_energy(g, ops, psi, chi1)
    E3 = axial_energy(g, ops, psi, [2.0 * b for b in chi1])
    assert abs(E2[0] - E[0]) <= 1e-10 * E[0]
    assert E2[1] > 0 and abs(E3[1] / E2[1] - 4.0) <= 1e-10
