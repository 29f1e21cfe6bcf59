"""Norms and integral diagnostics on the collocation nodes (oracle, FP64).

Area element under Eq. (1): r dr = ell^2 dx / (1 - x)^2, so a plane integral is
    int f r dr dphi dz  ~=  ell^2 sum_i w_i / (1 - x_i)^2 * (2 pi / Nphi) sum_j * (Lz / Nz) sum_l f.
* l2w(g, f): sqrt((1/Lz) int f^2 dA dz) on the nodes;
  weighted_l2(g, e, ref) = l2w(e) / l2w(ref), the relative weighted L2
  sqrt(sum w e^2/(1-x)^2) / sqrt(sum w ref^2/(1-x)^2) over all nodes (the uniform phi
  and z weights cancel).  This reading reproduces the relative errors of Table 2 to
  four digits.
* circulation / second_moment: Eq. (16) with the mapped quadrature.
"""

import math

import numpy as np


def _area_w(g):
    return g.w / (1.0 - g.x) ** 2


def l2w(g, f):
    """Plane-averaged area-weighted L2 norm sqrt((1/Lz) int f^2 dA dz) with the
    mapped quadrature (uniform phi and z weights)."""
    a = _area_w(g)[None, None, :]
    return math.sqrt(g.ell ** 2 * (2.0 * math.pi / g.nphi) * float(np.sum(a * f ** 2)) / g.nz)


def weighted_l2(g, err, ref):
    return l2w(g, err) / l2w(g, ref)


def circulation(g, omega):
    """Eq. (16) Gamma for a field [Nz][Nphi][Nr] (averaged over z)."""
    a = _area_w(g)[None, None, :]
    return g.ell ** 2 * (2.0 * math.pi / g.nphi) * float(np.sum(a * omega)) / g.nz


def second_moment(g, omega):
    a = (_area_w(g) * g.r ** 2)[None, None, :]
    return g.ell ** 2 * (2.0 * math.pi / g.nphi) * float(np.sum(a * omega)) / g.nz
