"""Oracle-built vortex states shared by the CPU pins and the GPU parity tests."""

import numpy as np

import oracle as O
from oracle import logproxy as LP
from oracle.vortex import VortexOps


def q_vortex_state(g, centres, q=1.0, ops=None):
    """(psi, chi, c_psi, c_chi, ops) of a sum of q-vortices (v_phi = (1 - e^{-rho^2}) / rho,
    v_z = e^{-rho^2} / q about each centre): omega_z = 2 e^{-rho^2} and v_z at the nodes,
    forward transforms, lap_h^{-1} per harmonic (lap psi = -w_z, lap chi = -v_z), the
    (0, 0) blocks solved for their log amplitudes (Sec. 3.1, Eq. (6))."""
    r, phi, z = g.nodes3()
    X, Y = r * np.cos(phi) + 0 * z, r * np.sin(phi) + 0 * z
    wz = np.zeros_like(X)
    vz = np.zeros_like(X)
    for (x0, y0) in centres:
        e = np.exp(-((X - x0) ** 2 + (Y - y0) ** 2))
        wz += 2.0 * e
        vz += e / q
    ops = ops or VortexOps(g)
    lam = LP.image(g.nc, g.ell)
    out, cs = [], []
    for f in (O.forward(g, -wz), O.forward(g, -vz)):
        s = [np.stack([ops.lap_h_inv(m, f[m][kk]) for kk in range(g.K)]) for m in range(g.M)]
        s[0][0], c = LP.solve_for_c(ops.D[0], lam, f[0][0])
        out.append(s)
        cs.append(c)
    return out[0], out[1], cs[0], cs[1], ops
