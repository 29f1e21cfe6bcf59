"""Helpers shared by the GPU parity tests: matched oracle grid and GPU context."""

import numpy as np

import oracle as O
from paper_2609_18026_b300 import binding as B
from paper_2609_18026_b300 import workloads as W


def pair(nr, nphi, nz, ell, lz=2 * np.pi, policy="linear", precision=B.FP64, **chops):
    g = O.Grid(nr, nphi, nz, ell, lz=lz, policy=policy,
               nr_c=chops.get("nr_c"), M=chops.get("nphi_c"), Kz=chops.get("nz_c"))
    ctx = B.Context(nr, nphi, nz, ell, lz=lz, precision=precision,
                    chop_policy={"linear": B.CHOP_LINEAR, "twothirds": B.CHOP_TWOTHIRDS,
                                 "nyquist": B.CHOP_NYQUIST}[policy],
                    nr_c=chops.get("nr_c") or 0, nphi_c=chops.get("nphi_c") or 0,
                    nz_c=chops.get("nz_c") or 0)
    assert (ctx.M, ctx.Kz, ctx.nc) == (g.M, g.Kz, g.nc)
    return g, ctx


def to_gpu_phys(ctx, arr):
    import torch
    return torch.as_tensor(np.ascontiguousarray(arr), dtype=ctx.phys_dtype).cuda()


def to_gpu_spec(flat):
    import torch
    return torch.as_tensor(np.ascontiguousarray(flat), dtype=torch.complex128).cuda()


def spec_from_gpu(g, t):
    return O.from_flat(g, t.cpu().numpy())


def rand_phys(g, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((g.nz, g.nphi, g.nr))


def rand_spec(g, seed):
    return W.random_spectral(g.nc, g.M, g.Kz, seed=seed)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def block_err(g, got, ref, floor=0.0):
    """Worst per-(m, k)-block relative error of two spectral lists:
    max over blocks of max|got - ref| / max(max|ref_block|, floor * max|ref|).
    With floor = 0 every block is held to its own scale, so a wrong coefficient
    in a block that is small in norm cannot hide behind the global norm."""
    gmax = max(float(np.max(np.abs(b))) for b in ref if b.size)
    worst = 0.0
    for a, b in zip(got, ref):
        for kk in range(b.shape[0]):
            d = float(np.max(np.abs(a[kk] - b[kk]))) if b.shape[1] else 0.0
            s = max(float(np.max(np.abs(b[kk]))) if b.shape[1] else 0.0, floor * gmax, 1e-300)
            worst = max(worst, d / s)
    return worst


def max_err(got, ref):
    """Element-wise bound: max|got - ref| / max|ref|."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(got - ref)) / max(float(np.max(np.abs(ref))), 1e-300))
