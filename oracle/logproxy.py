"""Logarithmic far-field proxy of a scalar with a nonzero planar integral (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 3.1, Eq. (6).  The basis functions all decay, so no combination of them
represents the logarithmic far field that a two-dimensional Poisson solution has
when its source integrates to a nonzero value.  A scalar therefore carries one
extra real amplitude c of the proxy Lambda(r) = ln(r^2 + ell^2):
    s = c Lambda + sum_{n,m,k} shat_nmk Pbar_n^m e^{i(m phi + kappa z)}.
The horizontal Laplacian of the proxy lies inside the basis:
    lap_h Lambda = (4/3 P_0 - 2 P_1 + 2/3 P_2) / ell^2 = (1 - x)^2 / ell^2
(unnormalised P_n = P_n^0 at x(r)).  Only the harmonic (m, k) = (0, 0) is affected.

* image(nc, ell): lam, the coefficients of lap_h Lambda on the normalised basis:
  Eq. (6) divided by N_n^0 = sqrt((2n + 1) / 2).
* lap_apply(D0, lam, s, c): the forward horizontal Laplacian of (s, c) in the (0, 0)
  block, D_0 s + c lam.  The result has no logarithmic part.
* solve_prescribed(D0, lam, f, c): inversion with c given.  D_0 s = f - c lam, with
  the singular first row of D_0 replaced by the far-field decay condition
  sum_n Pbar_n^0(1) s_n = 0 and right-hand side 0, the condition every c = 0 solve
  of the package uses.
* solve_for_c(D0, lam, f): inversion with c unknown.  The first column of D_0
  (zero: a constant has zero Laplacian) is replaced by lam.  The unknown in its
  place is c, and the Pbar_0^0 coefficient of s is zero.
* node_fields(r, ell, c_psi, c_chi): the velocity and vorticity of the proxies
  c_psi Lambda (toroidal) and c_chi Lambda (poloidal) in closed form at radii r,
  with the conventions v = curl(psi e_z) + curl curl(chi e_z):
      v_phi = -c_psi dLambda/dr   = -2 c_psi r / (r^2 + ell^2)
      w_z   = -c_psi lap_h Lambda = -4 c_psi ell^2 / (r^2 + ell^2)^2
      v_z   = -c_chi lap_h Lambda = -4 c_chi ell^2 / (r^2 + ell^2)^2
      w_phi =  c_chi d(lap_h Lambda)/dr = -16 c_chi ell^2 r / (r^2 + ell^2)^3
  (v_r = w_r = 0: the proxies are axisymmetric and z-independent).
* source(D0, lam, nu, nu_h, p): L Lambda, the dissipation operator of Eq. (11) at
  (m, k) = (0, 0) applied to the proxy, L = nu lap_h - nu_h (-lap_h)^{p/2}:
      L Lambda = nu lam - nu_h (-1)^{p/2} D_0^{p/2 - 1} lam.
  The proxy amplitudes are constant in time (the net circulation and the net axial
  flux of a decaying flow are conserved, so the projected nonlinear term has no
  logarithmic part), and the proxy enters the time step as the constant forcing
  c L Lambda of the (0, 0) block.

Readings (the paper gives the two inversion variants in one sentence each): the
prescribed-c variant keeps the decay-row gauge of the c = 0 solves for the basis
part, and the solve-for-c variant sets the Pbar_0^0 coefficient to zero, as the
paper's "the unknown multiplying P_0^0 becomes c" states.  The two results then
differ only in that coefficient, a constant that no velocity or vorticity sees.

Pins (tests/test_oracle_logproxy.py): the Lamb-Oseen stream function in closed
form (exponential integral) for both inversion variants and the amplitude
c = -Gamma / (4 pi); the forward Laplacian of the recovered pair against the
source; node fields against the Legendre forms the CUDA path adds; the
hyperviscous source against sympy's iterated Laplacian of (1 - x)^2 / ell^2; the
diffusing Lamb-Oseen vortex over time; a shifted q-vortex, a steady Euler flow
with net circulation and net axial flux, whose projected nonlinear term vanishes.
"""

import math

import numpy as np

from .basis import pbar_table


def image(nc, ell):
    """Normalised coefficients of lap_h Lambda (length nc)."""
    lam = np.zeros(nc)
    unnorm = (4.0 / 3.0, -2.0, 2.0 / 3.0)
    for n in range(min(3, nc)):
        lam[n] = unnorm[n] / math.sqrt((2 * n + 1) / 2.0) / (ell * ell)
    return lam


def lap_apply(D0, lam, s, c):
    return D0 @ s + c * lam


def _decay_row(nc):
    # Pbar_n^0(1) = N_n^0 P_n(1) = sqrt((2n + 1) / 2)
    return pbar_table(1, nc, np.array([1.0]))[0][:, 0]


def solve_prescribed(D0, lam, f, c):
    nc = D0.shape[0]
    A = D0.copy()
    A[0, :] = _decay_row(nc)
    b = np.array(f, dtype=np.complex128) - c * lam
    b[0] = 0.0
    return np.linalg.solve(A, b.real) + 1j * np.linalg.solve(A, b.imag)


def solve_for_c(D0, lam, f):
    """(s, c): s has a zero Pbar_0^0 coefficient.  f is the (0, 0) block of a real
    field, so only its real part carries the amplitude: c = Re(y_0), and the
    imaginary part's y_0 (zero for a real field) is dropped."""
    A = D0.copy()
    A[:, 0] = lam
    b = np.array(f, dtype=np.complex128)
    yr = np.linalg.solve(A, b.real)
    yi = np.linalg.solve(A, b.imag)
    c = float(yr[0])
    s = yr + 1j * yi
    s[0] = 0.0
    return s, c


def node_fields(r, ell, c_psi, c_chi):
    """dict of the proxies' v_phi, w_z, v_z, w_phi at radii r."""
    q = r * r + ell * ell
    return {"v_phi": -2.0 * c_psi * r / q,
            "w_z": -4.0 * c_psi * ell * ell / (q * q),
            "v_z": -4.0 * c_chi * ell * ell / (q * q),
            "w_phi": -16.0 * c_chi * ell * ell * r / (q * q * q)}


def source(D0, lam, nu, nu_h=0.0, p=8):
    out = nu * lam
    if nu_h != 0.0:
        v = lam.copy()
        for _ in range(p // 2 - 1):
            v = D0 @ v
        out = out - nu_h * (-1.0) ** (p // 2) * v
    return out
