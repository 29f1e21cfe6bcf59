"""Pins of the oracle's toroidal-poloidal vortex term (CPU only)."""

import math

import numpy as np

import oracle as O


def _grid():
    return O.Grid(40, 8, 8, 1.0, lz=2 * math.pi, policy="linear")


def _nodes(g):
    return g.nodes3()


def test_gradient_field_projects_to_zero():
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
    C = -kap * r ** 2 * f * np.cos(2 * phi) * np.sin(kap * z)   # r^2 N_z = r^2 d_z g
    psiN, chiN = ops.project(O.forward(g, A), O.forward(g, Bf), O.forward(g, C))
    scale = O.spec_norm(g, O.forward(g, f * np.cos(2 * phi) * np.cos(kap * z)))
    assert O.spec_norm(g, psiN) < 1e-9 * scale
    assert O.spec_norm(g, chiN) < 1e-9 * scale


def test_solenoidal_field_projects_back():
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
    r2vz = O.forward(g, r ** 2 * O.backward(g, vz))
    pN, cN = ops.project(rvp, rvr, r2vz)
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


def test_axisymmetric_vortex_has_no_projected_forcing():
    # A shielded axisymmetric vortex (psi = -e^{-r^2}, zero net circulation):
    # N = (v_phi w_z) e_r is a pure gradient, so P(N) = 0 (the steady Euler
    # balance of a columnar vortex).
    g = O.Grid(48, 4, 4, 1.0, lz=4.0)
    ops = O.VortexOps(g)
    r, phi, z = g.nodes3()
    psi = O.forward(g, -np.exp(-r ** 2) + 0 * phi + 0 * z)
    chi = [np.zeros_like(b) for b in psi]
    pN, cN = ops.nonlinear(psi, chi, U0=0.0)
    assert O.spec_norm(g, pN) < 1e-9 * O.spec_norm(g, psi)
    assert O.spec_norm(g, cN) < 1e-9 * O.spec_norm(g, psi)


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
