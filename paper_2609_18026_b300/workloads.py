"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the spectral method: each function evaluates an
analytic initial condition (or draws seeded noise) at node coordinates that the
caller passes in, in the physical layout [Nz][Nphi][Nr] (r fastest).  Random
numbers come from numpy's PCG64 with the seed stated per workload, so the CUDA
path and the oracle receive bit-identical inputs.

Workloads (all analytic, as in the paper's examples; no dataset is involved):
* gaussian_polar      -- 2-D polar diffusion seed exp(-r^2)(1 + 0.5 cos 2 phi)
* gaussian_polar_reg  -- its pole-regular variant exp(-r^2) + 0.5 r^2 exp(-r^2) cos 2 phi
* fkpp_seed           -- Fisher-KPP bump exp(-r^2/4)(1 + 0.01 xi), xi ~ U(-1, 1) per node
* oseen               -- Oseen vorticity, Eq. (14)
* heat_mode           -- manufactured heat mode, Eq. (15)
* field_sA / field_sB -- rational and Gaussian fields of Eq. (13)
* kpp_linear          -- linearised Fisher-KPP solution, Eq. (18)
* vortex_pair_omega   -- counter-rotating Lamb-Oseen pair with a seeded axial displacement
* q_vortex_pair       -- co-rotating q-vortex pair (axial vorticity and axial velocity)
* random_spectral     -- seeded random coefficients in the flat ragged layout
* batch_instances     -- the uneven batch of independent 2-D/3-D solves
* surrogate_trajectories -- seeded vortex-pair variants the learned surrogate trains on
"""

import math

import numpy as np


def _b(r, phi, z):
    return np.broadcast_arrays(r, phi, z)


def gaussian_polar(r, phi, z):
    r, phi, z = _b(r, phi, z)
    return np.exp(-r * r) * (1.0 + 0.5 * np.cos(2.0 * phi))


def gaussian_polar_reg(r, phi, z):
    r, phi, z = _b(r, phi, z)
    e = np.exp(-r * r)
    return e + 0.5 * r * r * e * np.cos(2.0 * phi)


def fkpp_seed(r, phi, z, seed=2, noise=0.01):
    r, phi, z = _b(r, phi, z)
    xi = np.random.Generator(np.random.PCG64(seed)).uniform(-1.0, 1.0, size=r.shape)
    return np.exp(-r * r / 4.0) * (1.0 + noise * xi)


def oseen(r, phi, z, t, nu=0.1, sigma0=1.0):
    r, phi, z = _b(r, phi, z)
    B = 1.0 + 2.0 * nu * t / sigma0 ** 2
    return np.exp(-r * r / (2.0 * sigma0 ** 2 * B)) / (2.0 * math.pi * sigma0 ** 2 * B)


def heat_mode(r, phi, z, t, m=2, nu=0.1, sigma0=1.0, A=1.0):
    r, phi, z = _b(r, phi, z)
    B = 1.0 + 2.0 * nu * t / sigma0 ** 2
    return (A * B ** (-(m + 1)) * (r / sigma0) ** m
            * np.exp(-r * r / (2.0 * sigma0 ** 2 * B)) * np.cos(m * phi))


def field_sA(r, phi, z, a=1.7):
    r, phi, z = _b(r, phi, z)
    q = r * r + a * a
    return r * np.cos(phi) / q + r * r * np.cos(2.0 * phi) / (q * q)


def field_sB(r, phi, z, sigma=1.0):
    r, phi, z = _b(r, phi, z)
    return (r / sigma) ** 2 * np.exp(-r * r / (2.0 * sigma ** 2)) * np.cos(2.0 * phi)


def kpp_linear(r, phi, z, t, A=1e-6, D=1.0, gamma=0.25, sigma=1.0):
    r, phi, z = _b(r, phi, z)
    s2 = sigma ** 2 + 2.0 * D * t
    return A * sigma ** 2 / s2 * math.exp(gamma * t) * np.exp(-r * r / (2.0 * s2))


def vortex_pair_omega(r, phi, z, lz, b=1.0, a=0.2, gamma=2.0 * math.pi, amp=1e-3, incl_deg=48.0, kseed=1):
    """Axial vorticity of two counter-rotating Lamb-Oseen vortices (circulations
    +-gamma, core radius a) at (x, y) = (-+b/2, 0), each displaced by
    amp cos(2 pi kseed z / lz) along a direction inclined incl_deg from the x axis,
    mirror-symmetric about x = 0."""
    r, phi, z = _b(r, phi, z)
    x = r * np.cos(phi)
    y = r * np.sin(phi)
    d = amp * np.cos(2.0 * math.pi * kseed * z / lz)
    th = math.radians(incl_deg)
    out = np.zeros_like(x)
    for sgn, xc in ((+1.0, -0.5 * b), (-1.0, 0.5 * b)):
        # mirror symmetry about x = 0: the x-displacement flips sign
        dx = d * math.cos(th) * (-1.0 if xc < 0 else 1.0)
        dy = d * math.sin(th)
        rr = (x - xc - dx) ** 2 + (y - dy) ** 2
        out += sgn * gamma / (math.pi * a * a) * np.exp(-rr / (a * a))
    return out


def q_vortex_pair(r, phi, z, lz, b=4.0, q=1.0, amp=1e-10, kseed=1):
    """(omega_z, v_z) of two co-rotating q-vortices (v_phi = (1 - e^{-rho^2}) / rho and
    v_z = e^{-rho^2} / q about each centre, so omega_z = 2 e^{-rho^2}) at (x, y) =
    (+-b/2, 0), each centre displaced along x by amp cos(2 pi kseed z / lz) in
    opposite directions (a deterministic seed of the given amplitude)."""
    r, phi, z = _b(r, phi, z)
    x = r * np.cos(phi)
    y = r * np.sin(phi)
    d = amp * np.cos(2.0 * math.pi * kseed * z / lz)
    wz = np.zeros_like(x)
    vz = np.zeros_like(x)
    for xc, sgn in ((0.5 * b, 1.0), (-0.5 * b, -1.0)):
        e = np.exp(-((x - xc - sgn * d) ** 2 + y ** 2))
        wz += 2.0 * e
        vz += e / q
    return wz, vz


def random_spectral(nc, M, Kz, seed=0, scale_decay=0.0):
    """Seeded complex coefficients in the flat ragged layout [m][k][n - m].

    The m = 0 block is made Hermitian in k (coefficient at -k is the conjugate of
    the one at +k, k = 0 real) so that it describes a real field.
    """
    K = 2 * Kz - 1
    rng = np.random.Generator(np.random.PCG64(seed))
    blocks = []
    for m in range(M):
        n = np.arange(m, nc)
        amp = np.exp(-scale_decay * n)
        blk = (rng.standard_normal((K, nc - m)) + 1j * rng.standard_normal((K, nc - m))) * amp[None, :]
        if m == 0:
            blk[0] = blk[0].real
            for k in range(1, Kz):
                blk[K - k] = np.conj(blk[k])
        blocks.append(blk.reshape(-1))
    return np.concatenate(blocks).astype(np.complex128)


def batch_instances(n=64, seed=20261202):
    """Parameters of the uneven batch: one dict per instance.

    Nr in {32,64,128,256}, Nphi in {16,32,64,128,256}, Nz in {1,16,64},
    ell ~ U[0.5, 4], kind diffusion (nu = 1e-2) or Fisher-KPP (D = 1, gamma = 1)
    with probability 1/2, an off-centre Gaussian of width sigma ~ U[0.5, 2] ell
    centred at (x0, y0) uniform in [-ell, ell]^2.  Lz = 2 pi, dt = 1e-3.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        nr = int(rng.choice([32, 64, 128, 256]))
        nphi = int(rng.choice([16, 32, 64, 128, 256]))
        nz = int(rng.choice([1, 16, 64]))
        ell = float(rng.uniform(0.5, 4.0))
        kind = "fkpp" if rng.uniform() < 0.5 else "diffusion"
        sigma = float(rng.uniform(0.5, 2.0)) * ell
        x0 = float(rng.uniform(-ell, ell))
        y0 = float(rng.uniform(-ell, ell))
        out.append(dict(index=i, nr=nr, nphi=nphi, nz=nz, ell=ell, kind=kind,
                        sigma=sigma, x0=x0, y0=y0, lz=2.0 * math.pi, dt=1e-3))
    return out


def batch_initial(inst, r, phi, z):
    """Off-centre Gaussian of one batch instance (times an axial modulation in 3-D)."""
    r, phi, z = _b(r, phi, z)
    X = r * np.cos(phi) - inst["x0"]
    Y = r * np.sin(phi) - inst["y0"]
    f = np.exp(-(X * X + Y * Y) / (2.0 * inst["sigma"] ** 2))
    if inst["nz"] > 1:
        f = f * (1.0 + 0.1 * np.cos(2.0 * math.pi * z / inst["lz"]))
    return f


def surrogate_trajectories(n=2000, seed=20261203):
    """Seeded parameters of the vortex-pair trajectories for the learned surrogate.

    Per trajectory: axial displacement amplitude 1e-3 x U[0.5, 2], perturbation-plane
    inclination U[40, 56] degrees, separation b ~ U[0.9, 1.1], core radius
    a ~ U[0.18, 0.22]; circulation 2 pi and one axial wavelength as in
    vortex_pair_omega."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        amp = 1e-3 * float(rng.uniform(0.5, 2.0))
        incl = float(rng.uniform(40.0, 56.0))
        b = float(rng.uniform(0.9, 1.1))
        a = float(rng.uniform(0.18, 0.22))
        out.append(dict(index=i, amp=amp, incl_deg=incl, b=b, a=a))
    return out
