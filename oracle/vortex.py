"""Toroidal-poloidal vortex nonlinear term (oracle, FP64).

Sec. 3.2 and Eq. (19): a solenoidal field V = curl(psi e_z) + curl curl(chi e_z)
(Eq. (8)) evolves as d(psi, chi)/dt = P[(U + v) x omega] + L(psi, chi), with P the
toroidal-poloidal projection recovered from the two planar Poisson problems of
Eq. (9), grad_h^2 chi = -V_z and grad_h^2 psi = -(curl V)_z, inverted with the
banded Laplacian of Sec. 3.1.  The paper says neither how the vector components
are transformed nor how the right-hand sides of Eq. (9) are formed from a field
N that also carries a gradient part (Sec. 3.2: the projection removes it).  The
definition taken here works harmonic by harmonic, e^{i(m phi + kappa z)}:

Operators on the orthonormal coefficients of order m (n = m..Nc-1):
  R  = r d/dr (tridiagonal, Sec. 3.1),  D_m = horizontal Laplacian (Eq. (5)),
  J  = multiplication by x (the Jacobi matrix: x Pbar_n = a_{n+1} Pbar_{n+1} + a_n Pbar_{n-1},
       a_n = sqrt((n^2 - m^2)/(4 n^2 - 1))).
All products of truncated matrices (truncate, then compose).

velocity (from Eq. (8))      r v_r   = i m psi + i kappa R chi
                             r v_phi = -R psi - m kappa chi
                             v_z     = -D_m chi
vorticity (curl of Eq. (8):  omega = curl(Psi e_z) + curl curl(psi e_z),
           toroidal Psi = -(D_m - kappa^2) chi)
                             r w_r   = i m Psi + i kappa R psi
                             r w_phi = -R Psi - m kappa psi
                             w_z     = -D_m psi

project_plain (the oracle's definition of P; `nonlinear` uses it):
  1. Six backward transforms of the fields above; at the nodes divide the
     r-weighted ones by r_i, add the uniform background U = U0 e_y
     (U_r = U0 sin phi, U_phi = U0 cos phi; Sec. 5.3 moving frame) and form the
     primitive N = (v + U) x omega.
  2. A = r N_phi, B = r N_r and N_z at the nodes; three forward transforms.
  3. X1 = R A - i m B (= r^2 (curl N)_z) and X2 = R B + i m A (= r^2 div_h N).
  4. Two backward transforms, division by r_i^2 at the nodes, two forward
     transforms: (curl N)_z and div_h N; then div N = div_h N + i kappa N_z.
  5. psi_N = -lap_h^{-1} (curl N)_z  (Eq. (9));
     k != 0: g = (D_m - kappa^2)^{-1} div N and chi_N = -lap_h^{-1} (N_z - i kappa g);
     k == 0: chi_N = -lap_h^{-1} N_z.
     N = curl(psi_N e_z) + curl curl(chi_N e_z) + grad g is then the Helmholtz
     split of N, so the gradient part is removed (Sec. 3.2).
  13 transforms per evaluation.

project_banded (a second form; it is the formulation the CUDA path runs): the
same P with every step kept in coefficient space, so that nothing is divided by
r at the nodes.  With Q = (I - J^2) diag(-n(n+1)) = r^2 grad_h^2 (from Eq. (3):
r^2 grad_h^2 Pbar_n = -n(n+1)(1-x^2) Pbar_n) and (1 - x) r^2 = ell^2 (1 + x)
(Eq. (1)), the products are transformed as A = r N_phi, B = r N_r, C = r^2 N_z
(9 transforms per evaluation) and
    Q psi_N = -X1                                                   (lap_h psi_N = -(curl N)_z, times r^2)
    [(I - J) Q - kappa^2 ell^2 (I + J)] g = (I - J)(X2 + i kappa C)   (k != 0; (lap_h - kappa^2) g = div N, times (1-x) r^2)
    (I - J) Q chi_N = i kappa ell^2 (I + J) g - (I - J) C           (lap_h chi_N = i kappa g - N_z, times (1-x) r^2)
(g = 0 at k = 0).  The two forms agree in exact arithmetic; on a truncated
expansion they differ by the truncation of the products, which falls
spectrally with Nr for resolved fields (pinned in tests/test_oracle_vortex.py).

At m = 0 the horizontal Laplacian (and Q, (I - J) Q) has a zero first column (the
constant has zero Laplacian); its first row is replaced by the far-field decay
condition sum_n Pbar_n^0(1) s_n = 0 with right-hand side 0 (log-proxy coefficient
c = 0, Sec. 3.1 / Eq. (6): exact for the zero-net-circulation vortex pair).
The inverse horizontal Laplacian with the same decay row (lap_h_inv) gives the
initial stream function psi = -lap_h^{-1} omega_z of a vortex workload.

Pins (tests/test_oracle_vortex.py): J against Gauss quadrature of <Pbar_j, x Pbar_n>;
Q against quadrature of <Pbar_j, r^2 lap_h Pbar_n>; for both forms: gradient fields
project to zero, a solenoidal field built from known (psi, chi) projects back to
them, an axisymmetric shielded vortex has a pure-gradient N so P(N) = 0, and in a
uniform background U0 e_y its projected forcing is the translation
psi_N = -U0 d(psi)/dy in closed form; analytic curl fields; the decay-row Laplacian
inverse; plain and banded forms agree to a bound that falls spectrally with Nr;
the axial energy spectrum (axial_energy) of a shielded axisymmetric vortex against
its closed form.
The full nonlinear evolution is checked against the oracle only: parity unpinned
beyond these properties.
"""

import math

import numpy as np
import scipy.linalg as sla

from . import logproxy
from .operators import del2h_closed, rdr_matrix
from .transform import backward, forward, serial


def jacobi_matrix(m, nc):
    """Multiplication by x on the orthonormal order-m coefficients (tridiagonal),
    from x Pbar_n^m = a_{n+1} Pbar_{n+1}^m + a_n Pbar_{n-1}^m, a_n = sqrt((n^2-m^2)/(4n^2-1))."""
    N = nc - m
    J = np.zeros((N, N))
    for a in range(N - 1):
        n = m + a + 1
        v = math.sqrt((n * n - m * m) / (4.0 * n * n - 1.0))
        J[a, a + 1] = v
        J[a + 1, a] = v
    return J


def pbar_at_one(m, nc):
    """Pbar_n^m(1): sqrt((2n+1)/2) for m = 0, zero otherwise."""
    if m != 0:
        return np.zeros(nc - m)
    n = np.arange(0, nc)
    return np.sqrt((2.0 * n + 1.0) / 2.0)


class VortexOps:
    """Band operators and solvers of the toroidal-poloidal formulation."""

    def __init__(self, g):
        with serial():
            self._setup(g)

    def _setup(self, g):
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
        # banded projection operators
        self.J, self.Q, self.H = [], [], []
        self.lu_Q, self.lu_H = [], []
        for m in range(g.M):
            J = jacobi_matrix(m, g.nc)
            n = np.arange(m, g.nc, dtype=np.float64)
            I = np.eye(g.nc - m)
            Q = (I - J @ J) @ np.diag(-n * (n + 1.0))
            H = (I - J) @ Q
            self.J.append(J)
            self.Q.append(Q)
            self.H.append(H)
            Qd, Hd = Q.copy(), H.copy()
            if m == 0:
                Qd[0, :] = pbar_at_one(0, g.nc)
                Hd[0, :] = pbar_at_one(0, g.nc)
            self.lu_Q.append(sla.lu_factor(Qd))
            self.lu_H.append(sla.lu_factor(Hd))
        # (D_m - kappa^2) per (m, |k|), |k| >= 1 (nonsingular: no decay row)
        self.lu_helm = {}
        for m in range(g.M):
            I = np.eye(g.nc - m)
            for kabs in range(1, g.Kz):
                kappa = 2.0 * math.pi * kabs / g.lz
                self.lu_helm[(m, kabs)] = sla.lu_factor(self.D[m] - kappa * kappa * I)
        self.lu_G = {}
        for m in range(g.M):
            I = np.eye(g.nc - m)
            for kabs in range(1, g.Kz):
                kappa = 2.0 * math.pi * kabs / g.lz
                G = self.H[m] - kappa * kappa * g.ell ** 2 * (I + self.J[m])
                self.lu_G[(m, kabs)] = sla.lu_factor(G)

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

    @staticmethod
    def _csolve(lu, rhs):
        return sla.lu_solve(lu, rhs.real) + 1j * sla.lu_solve(lu, rhs.imag)

    def _decay_solve(self, lu, m, rhs):
        b = np.array(rhs, dtype=np.complex128)
        if m == 0:
            b[0] = 0.0
        return self._csolve(lu, b)

    def fields(self, psi, chi):
        """Spectral (r v_r, r v_phi, v_z, r w_r, r w_phi, w_z) from (psi, chi)."""
        with serial():
            return self._fields(psi, chi)

    def _fields(self, psi, chi):
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

    def _nodes(self):
        g = self.g
        return g.r[None, None, :], g.phi[None, :, None]

    # ---------------- the oracle's definition: project_plain (13 transforms)
    def primitive_fields(self, psi, chi, cpsi=0.0, cchi=0.0):
        """(v_r, v_phi, v_z, w_r, w_phi, w_z) at the nodes: six backward transforms
        of the spectral fields, the division by r at the nodes, and the velocity and
        vorticity of the log proxies c_psi Lambda, c_chi Lambda in closed form."""
        g = self.g
        rvr, rvp, vz, rwr, rwp, wz = (backward(g, f) for f in self.fields(psi, chi))
        r, _ = self._nodes()
        lp = logproxy.node_fields(r, g.ell, cpsi, cchi)
        return (rvr / r, rvp / r + lp["v_phi"], vz + lp["v_z"],
                rwr / r, rwp / r + lp["w_phi"], wz + lp["w_z"])

    def products_plain(self, psi, chi, U0=0.0, Uz=0.0, cpsi=0.0, cchi=0.0):
        """Spectral (A, B, Nz) = (r N_phi, r N_r, N_z) of N = (U + v) x omega with
        U = U0 e_y + Uz e_z, formed from the primitive components at the nodes
        (steps 1-2 above)."""
        g = self.g
        vr, vp, vz, wr, wp, wz = self.primitive_fields(psi, chi, cpsi, cchi)
        r, phi = self._nodes()
        vr = vr + U0 * np.sin(phi)             # v_r + U_r
        vp = vp + U0 * np.cos(phi)             # v_phi + U_phi
        vz = vz + Uz                           # v_z + U_z
        Nr = vp * wz - vz * wp
        Np = vz * wr - vr * wz
        Nz = vr * wp - vp * wr
        return forward(g, r * Np), forward(g, r * Nr), forward(g, Nz)

    def project_plain(self, A, Bf, Nz):
        """P of the field with spectral r N_phi = A, r N_r = B and N_z (steps 3-5)."""
        g = self.g
        X1 = [np.empty_like(A[m]) for m in range(g.M)]
        X2 = [np.empty_like(A[m]) for m in range(g.M)]
        with serial():
            for m in range(g.M):
                R = self.R[m]
                for kk in range(g.K):
                    X1[m][kk] = R @ A[m][kk] - 1j * m * Bf[m][kk]
                    X2[m][kk] = R @ Bf[m][kk] + 1j * m * A[m][kk]
        r, _ = self._nodes()
        curl_z = forward(g, backward(g, X1) / (r * r))
        div_h = forward(g, backward(g, X2) / (r * r))
        with serial():
            return self._plain_solves(curl_z, div_h, Nz)

    def _plain_solves(self, curl_z, div_h, Nz):
        g = self.g
        psiN, chiN = [], []
        for m in range(g.M):
            pb = np.empty((g.K, g.nc - m), dtype=np.complex128)
            cb = np.empty_like(pb)
            for kk in range(g.K):
                kap = self.kappa(kk)
                pb[kk] = -self.lap_h_inv(m, curl_z[m][kk])
                if g.kz[kk] != 0:
                    divN = div_h[m][kk] + 1j * kap * Nz[m][kk]
                    gg = self._csolve(self.lu_helm[(m, abs(int(g.kz[kk])))], divN)
                    cb[kk] = -self.lap_h_inv(m, Nz[m][kk] - 1j * kap * gg)
                else:
                    cb[kk] = -self.lap_h_inv(m, Nz[m][kk])
            psiN.append(pb)
            chiN.append(cb)
        return psiN, chiN

    def nonlinear_plain(self, psi, chi, U0=0.0, Uz=0.0, cpsi=0.0, cchi=0.0):
        return self.project_plain(*self.products_plain(psi, chi, U0, Uz, cpsi, cchi))

    # ---------------- the second form: project_banded (9 transforms)
    def products_banded(self, psi, chi, U0=0.0, Uz=0.0, cpsi=0.0, cchi=0.0):
        """Spectral (A, B, C) = (r N_phi, r N_r, r^2 N_z) of N = (U + v) x omega,
        formed from the r-weighted fields without division by r (the proxies'
        r-weighted fields in closed form at the nodes)."""
        g = self.g
        rvr, rvp, vz, rwr, rwp, wz = (backward(g, f) for f in self.fields(psi, chi))
        r, phi = self._nodes()
        lp = logproxy.node_fields(r, g.ell, cpsi, cchi)
        rvp = rvp + r * lp["v_phi"]
        vz = vz + lp["v_z"] + Uz
        rwp = rwp + r * lp["w_phi"]
        wz = wz + lp["w_z"]
        ar = rvr + r * U0 * np.sin(phi)       # r (v_r + U_r)
        ap = rvp + r * U0 * np.cos(phi)       # r (v_phi + U_phi)
        A = vz * rwr - ar * wz
        Bn = ap * wz - vz * rwp
        C = ar * rwp - ap * rwr
        return forward(g, A), forward(g, Bn), forward(g, C)

    def project_banded(self, A, Bf, C):
        """P of the field with spectral r N_phi = A, r N_r = B, r^2 N_z = C."""
        with serial():
            return self._project_banded(A, Bf, C)

    def _project_banded(self, A, Bf, C):
        g = self.g
        psiN, chiN = [], []
        for m in range(g.M):
            R, J = self.R[m], self.J[m]
            I = np.eye(g.nc - m)
            pb = np.empty((g.K, g.nc - m), dtype=np.complex128)
            cb = np.empty_like(pb)
            for kk in range(g.K):
                kap = self.kappa(kk)
                X1 = R @ A[m][kk] - 1j * m * Bf[m][kk]
                X2 = R @ Bf[m][kk] + 1j * m * A[m][kk]
                pb[kk] = self._decay_solve(self.lu_Q[m], m, -X1)
                if g.kz[kk] != 0:
                    kabs = abs(int(g.kz[kk]))
                    gg = self._csolve(self.lu_G[(m, kabs)], (I - J) @ (X2 + 1j * kap * C[m][kk]))
                    rhs = 1j * kap * g.ell ** 2 * ((I + J) @ gg) - (I - J) @ C[m][kk]
                else:
                    rhs = -((I - J) @ C[m][kk])
                cb[kk] = self._decay_solve(self.lu_H[m], m, rhs)
            psiN.append(pb)
            chiN.append(cb)
        return psiN, chiN

    def nonlinear_banded(self, psi, chi, U0=0.0, Uz=0.0, cpsi=0.0, cchi=0.0):
        return self.project_banded(*self.products_banded(psi, chi, U0, Uz, cpsi, cchi))

    def nonlinear(self, psi, chi, U0=0.0, form="plain", Uz=0.0, cpsi=0.0, cchi=0.0):
        """P[(U + v) x omega] for the state (psi, chi) with log-proxy amplitudes
        (cpsi, cchi) and background U = U0 e_y + Uz e_z; form "plain" (the
        definition) or "banded"."""
        if form == "plain":
            return self.nonlinear_plain(psi, chi, U0, Uz, cpsi, cchi)
        if form == "banded":
            return self.nonlinear_banded(psi, chi, U0, Uz, cpsi, cchi)
        raise ValueError(form)


def vortex_nonlinear(g, U0=0.0, form="plain", Uz=0.0, cpsi=0.0, cchi=0.0, source=None):
    """Nonlinear term for a two-field state [psi blocks..., chi blocks...] (2M blocks).

    With log proxies, source = (nu, nu_h, p) adds the proxies' constant forcing
    (cpsi, cchi) L Lambda to the (m, k) = (0, 0) blocks, so that a Stepper built
    with this term advances (psi, chi) with c Lambda included (see logproxy.py)."""
    ops = VortexOps(g)
    src = None
    if source is not None and (cpsi != 0.0 or cchi != 0.0):
        lam = logproxy.image(g.nc, g.ell)
        src = logproxy.source(ops.D[0], lam, *source)

    def A(state):
        psi, chi = state[:g.M], state[g.M:]
        pN, cN = ops.nonlinear(psi, chi, U0, form, Uz, cpsi, cchi)
        if src is not None:
            pN[0] = pN[0].copy()
            cN[0] = cN[0].copy()
            pN[0][0] += cpsi * src
            cN[0][0] += cchi * src
        return pN + cN
    return A, ops


def enstrophy(g, ops, psi, chi, cpsi=0.0, cchi=0.0):
    """(Z, w_max): Z = (1/2) int |omega|^2 dV over one axial period and the largest
    |omega| over the nodes, from the primitive vorticity at the nodes (the proxies'
    included), the mapped area quadrature r dr = ell^2 dx / (1 - x)^2, the uniform
    phi and z rules.  The paper reports enstrophy without defining its factor; the
    reading taken is the one half of the usual definition (Sec. 5.3)."""
    _, _, _, wr, wp, wz = ops.primitive_fields(psi, chi, cpsi, cchi)
    w2 = wr * wr + wp * wp + wz * wz
    a = g.w * g.ell ** 2 / (1.0 - g.x) ** 2
    Z = 0.5 * (g.lz / g.nz) * (2.0 * math.pi / g.nphi) * float(np.sum(w2 * a[None, None, :]))
    return Z, float(np.sqrt(np.max(w2)))


def axial_energy(g, ops, psi, chi):
    """Kinetic energy per axial wavenumber |k| of the velocity of (psi, chi), Eq. (8):
    E_|k| = (1/2) int |v_{+k}|^2 + |v_{-k}|^2 dV over one axial period, with v_k the
    k-th axial Fourier component of v (E_0: the k = 0 part alone), so that
    sum_|k| E_|k| = (1/2) int |v|^2 dV.  v = (r v_r / r, r v_phi / r, v_z) at the nodes
    (six backward transforms of the fields), the axial DFT along z, the mapped
    area quadrature r dr = ell^2 dx / (1 - x)^2 and the uniform phi rule."""
    rvr, rvp, vz = (backward(g, f) for f in ops.fields(psi, chi)[:3])
    r = g.r[None, None, :]
    v = [rvr / r, rvp / r, vz]
    a = g.w / (1.0 - g.x) ** 2
    E = np.zeros(g.nz // 2 + 1)
    for comp in v:
        vh = np.fft.fft(comp, axis=0) / g.nz                     # [k][phi][r]
        dens = np.sum(np.abs(vh) ** 2 * a[None, None, :], axis=(1, 2))   # sum over phi and the radial rule
        for k in range(g.nz):
            kk = k if k <= g.nz // 2 else g.nz - k
            E[kk] += dens[k]
    # (1/2) Lz * ell^2 * (2 pi / Nphi) * sum
    return 0.5 * g.lz * g.ell ** 2 * (2.0 * math.pi / g.nphi) * E[:g.Kz]
