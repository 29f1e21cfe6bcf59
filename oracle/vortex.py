"""Toroidal-poloidal vortex nonlinear term (oracle, FP64).

Sec. 3.2 and Eq. (19): a solenoidal field V = curl(psi e_z) + curl curl(chi e_z)
(Eq. (8)) evolves as d(psi, chi)/dt = P[(U + v) x omega] + L(psi, chi), with P the
toroidal-poloidal projection recovered from Eq. (9).  The paper does not spell out
how the vector components are transformed; the reading taken (identical in the
oracle and the CUDA path) works harmonic by harmonic, e^{i(m phi + kappa z)}, with
the banded r d/dr (R) and horizontal Laplacian (D_m) of Sec. 3.1:

velocity (from Eq. (8))      r v_r   = i m psi + i kappa R chi
                             r v_phi = -R psi - m kappa chi
                             v_z     = -D_m chi
vorticity (curl of Eq. (8):  omega = curl(Psi e_z) + curl curl(psi e_z),
           toroidal Psi = -(D_m - kappa^2) chi)
                             r w_r   = i m Psi + i kappa R psi
                             r w_phi = -R Psi - m kappa psi
                             w_z     = -D_m psi
At the nodes (six backward transforms): N = (v + U) x omega with the uniform
background U = U0 e_y (U_r = U0 sin phi, U_phi = U0 cos phi; Sec. 5.3 moving frame),
    A = r N_phi = v_z (r w_r) - (r v_r + r U_r) w_z
    B = r N_r   = (r v_phi + r U_phi) w_z - v_z (r w_phi)
    N_z = [(r v_r + r U_r)(r w_phi) - (r v_phi + r U_phi)(r w_r)] / r^2
Three forward transforms, then in spectral space
    X1 = R A - i m B   (= r^2 (curl N)_z),     X2 = R B + i m A   (= r^2 div_h N)
two backward transforms, division by r^2 at the nodes, two forward transforms give
(curl N)_z and div_h N; div N = div_h N + i kappa N_z.  Projection (Eq. (9) applied
to the solenoidal part of N = curl(psi_N e_z) + curl curl(chi_N e_z) + grad g):
    psi_N = -D_m^{-1} (curl N)_z
    g     = (D_m - kappa^2)^{-1} div N                  (k != 0)
    chi_N = -D_m^{-1} (N_z - i kappa g)                 (N_z alone when k == 0)
D_m is singular at m = 0 (the constant has zero Laplacian); there the first row is
replaced by the far-field decay condition sum_n Pbar_n^0(1) s_n = 0 with right-hand
side 0 (log-proxy coefficient c = 0, Sec. 3.1 / Eq. (6): exact for the zero-net-
circulation vortex pair).

Pins (tests/test_oracle_vortex.py): gradient fields project to zero; a solenoidal
field built from known (psi, chi) projects back to them; an axisymmetric Lamb-Oseen
vortex has a pure-gradient N so P(N) = 0; curl/divergence identities checked
against analytic fields.  The full nonlinear evolution is checked against the
oracle only: parity unpinned beyond these properties.
"""

import math

import numpy as np
import scipy.linalg as sla

from .operators import del2h_closed, rdr_matrix
from .transform import backward, forward


def pbar_at_one(m, nc):
    """Pbar_n^m(1): sqrt((2n+1)/2) for m = 0, zero otherwise."""
    if m != 0:
        return np.zeros(nc - m)
    n = np.arange(0, nc)
    return np.sqrt((2.0 * n + 1.0) / 2.0)


class VortexOps:
    """Band operators and solvers of the toroidal-poloidal formulation."""

    def __init__(self, g):
        self.g = g
        self.D = [del2h_closed(m, g.nc, g.ell) for m in range(g.M)]
        self.R = [rdr_matrix(m, g.nc) for m in range(g.M)]
        # D_m with the decay row at m = 0, LU once per m
        self.lu_h = []
        for m in range(g.M):
            Dm = self.D[m].copy()
            if m == 0:
                Dm[0, :] = pbar_at_one(0, g.nc)
            self.lu_h.append(sla.lu_factor(Dm))
        self.lu_helm = {}
        for m in range(g.M):
            for kabs in range(1, g.Kz):
                kappa = 2.0 * math.pi * kabs / g.lz
                self.lu_helm[(m, kabs)] = sla.lu_factor(self.D[m] - kappa * kappa * np.eye(g.nc - m))

    def kappa(self, kidx):
        return float(self.g.kappa[kidx])

    def lap_h_inv(self, m, rhs):
        """Solve D_m x = rhs (rhs a complex vector); m = 0 uses the decay row."""
        b = np.array(rhs, dtype=np.complex128)
        if m == 0:
            b[0] = 0.0
        xr = sla.lu_solve(self.lu_h[m], b.real)
        xi = sla.lu_solve(self.lu_h[m], b.imag)
        return xr + 1j * xi

    def helm_inv(self, m, kidx, rhs):
        kabs = abs(int(self.g.kz[kidx]))
        lu = self.lu_helm[(m, kabs)]
        return sla.lu_solve(lu, rhs.real) + 1j * sla.lu_solve(lu, rhs.imag)

    def fields(self, psi, chi):
        """Spectral (r v_r, r v_phi, v_z, r w_r, r w_phi, w_z) from (psi, chi)."""
        g = self.g
        out = [[None] * g.M for _ in range(6)]
        for m in range(g.M):
            D, R = self.D[m], self.R[m]
            rvr = np.empty((g.K, g.nc - m), dtype=np.complex128)
            rvp, vz, rwr, rwp, wz = (np.empty_like(rvr) for _ in range(5))
            for kk in range(g.K):
                kap = self.kappa(kk)
                p, c = psi[m][kk], chi[m][kk]
                Psi = -(D @ c - kap * kap * c)
                rvr[kk] = 1j * m * p + 1j * kap * (R @ c)
                rvp[kk] = -(R @ p) - m * kap * c
                vz[kk] = -(D @ c)
                rwr[kk] = 1j * m * Psi + 1j * kap * (R @ p)
                rwp[kk] = -(R @ Psi) - m * kap * p
                wz[kk] = -(D @ p)
            for f, v in enumerate((rvr, rvp, vz, rwr, rwp, wz)):
                out[f][m] = v
        return out

    def project(self, A, Bf, Nz):
        """P of the field with spectral r N_phi = A, r N_r = B, N_z = Nz."""
        g = self.g
        X1, X2 = [], []
        for m in range(g.M):
            R = self.R[m]
            X1.append(np.stack([R @ A[m][kk] - 1j * m * Bf[m][kk] for kk in range(g.K)]))
            X2.append(np.stack([R @ Bf[m][kk] + 1j * m * A[m][kk] for kk in range(g.K)]))
        inv_r2 = (1.0 / g.r ** 2)[None, None, :]
        curlz = forward(g, backward(g, X1) * inv_r2)
        divh = forward(g, backward(g, X2) * inv_r2)
        psiN, chiN = [], []
        for m in range(g.M):
            pb = np.empty((g.K, g.nc - m), dtype=np.complex128)
            cb = np.empty_like(pb)
            for kk in range(g.K):
                kap = self.kappa(kk)
                pb[kk] = -self.lap_h_inv(m, curlz[m][kk])
                if g.kz[kk] != 0:
                    divN = divh[m][kk] + 1j * kap * Nz[m][kk]
                    gg = self.helm_inv(m, kk, divN)
                    cb[kk] = -self.lap_h_inv(m, Nz[m][kk] - 1j * kap * gg)
                else:
                    cb[kk] = -self.lap_h_inv(m, Nz[m][kk])
            psiN.append(pb)
            chiN.append(cb)
        return psiN, chiN

    def nonlinear(self, psi, chi, U0=0.0):
        """P[(U + v) x omega] for the state (psi, chi)."""
        g = self.g
        sf = self.fields(psi, chi)
        rvr, rvp, vz, rwr, rwp, wz = (backward(g, f) for f in sf)
        r = g.r[None, None, :]
        phi = g.phi[None, :, None]
        rUr = r * U0 * np.sin(phi)
        rUp = r * U0 * np.cos(phi)
        ar = rvr + rUr
        ap = rvp + rUp
        A = vz * rwr - ar * wz
        Bn = ap * wz - vz * rwp
        Nz = (ar * rwp - ap * rwr) / (r * r)
        return self.project(forward(g, A), forward(g, Bn), forward(g, Nz))


def vortex_nonlinear(g, U0=0.0):
    """Nonlinear term for a two-field state [psi blocks..., chi blocks...] (2M blocks)."""
    ops = VortexOps(g)

    def A(state):
        psi, chi = state[:g.M], state[g.M:]
        pN, cN = ops.nonlinear(psi, chi, U0)
        return pN + cN
    return A, ops
