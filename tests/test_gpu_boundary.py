"""Boundary calls beyond the transforms: integral diagnostics (mlx_diag),
checkpoint images (mlx_get_state / mlx_set_state) and the device status word's
non-finite flag (MLX_ENUMERIC) of the nonlinear kernels."""

import math

import numpy as np
import pytest

import oracle as O
from paper_2609_18026_b300 import binding as B
from paper_2609_18026_b300 import workloads as W

from gpu_common import pair, to_gpu_spec, spec_from_gpu, rand_spec

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [B.FP64, B.BF16X3])
@pytest.mark.parametrize("grid", [(96, 4, 1, 1.0, "linear"), (40, 16, 8, 1.5, "twothirds")])
def test_diag_against_oracle(grid, prec, record):
    # Oseen vorticity (Eq. (14)): Gamma = 1, M2 of Table 2; and a random 3-D field
    nr, nphi, nz, ell, pol = grid
    g, ctx = pair(nr, nphi, nz, ell, lz=3.0, policy=pol, precision=prec, **({"nphi_c": 1} if nphi == 4 else {}))
    r, phi, z = g.nodes3()
    fields = [O.forward(g, W.oseen(r, phi, z, 0.0) + 0 * phi + 0 * z), O.from_flat(g, rand_spec(g, 3))]
    a = g.w / (1.0 - g.x) ** 2
    u64 = 2.0 ** -53
    for s in fields:
        u = O.backward(g, s)
        ref = dict(integral=O.circulation(g, u), moment2=O.second_moment(g, u), l2w=O.l2w(g, u),
                   spec_l2=O.spec_norm(g, s))
        got = ctx.diag(to_gpu_spec(O.to_flat(g, s)))
        # Rounding bound of the two quadrature sums, for either evaluation order:
        # f_00(x_i) = sum_n Pbar_n(x_i) s_n carries at most Nc u sum_n |Pbar_n s_n|,
        # weighted by a_i = w_i/(1-x_i)^2 (times r_i^2) - up to 1e8 at the last
        # nodes, so the far field's cancellation dominates; the node sum adds Nr u.
        absf = np.abs(g.P[0]).T @ np.abs(s[0][0])          # sum_n |Pbar_n(x_i) s_n| per node
        c = 2 * np.pi * g.ell ** 2
        bound = {"integral": c * (g.nc + g.nr) * u64 * float(np.sum(a * absf)),
                 "moment2": c * (g.nc + g.nr) * u64 * float(np.sum(a * g.r ** 2 * absf)),
                 "l2w": 1e-12 * ref["l2w"], "spec_l2": 1e-12 * ref["spec_l2"]}
        errs = {k: abs(got[k] - ref[k]) for k in ref}
        record("diag", grid=grid[:3], precision=prec, **{k: errs[k] / (abs(ref[k]) or 1.0) for k in ref},
               moment2_bound=bound["moment2"] / abs(ref["moment2"] or 1.0))
        for k in ref:
            assert errs[k] <= 1e-12 * abs(ref[k]) + 2.0 * bound[k], (k, got[k], ref[k], bound[k])
    # the Oseen vortex at t = 0 has unit circulation (Eq. (14))
    assert abs(ctx.diag(to_gpu_spec(O.to_flat(g, fields[0])))["integral"] - 1.0) < 1e-6


@pytest.mark.parametrize("kind", [B.NONLIN_FKPP, B.NONLIN_VORTEX])
def test_checkpoint_image_resume_bitwise(kind):
    # N steps == k steps, image, a fresh context restores it, N - k steps: bitwise
    import torch
    nr, nphi, nz, ell, lz = 24, 16, 8, 1.0 if kind == B.NONLIN_VORTEX else 4.0, 8.6
    g, a_ctx = pair(nr, nphi, nz, ell, lz=lz, policy="twothirds")
    _, b_ctx = pair(nr, nphi, nz, ell, lz=lz, policy="twothirds")
    nf = 2 if kind == B.NONLIN_VORTEX else 1
    for c in (a_ctx, b_ctx):
        if kind == B.NONLIN_VORTEX:
            c.vortex_setup()
            c.implicit_setup(1e-3, 1e-3, nu_h=5e-7, p=8)
        else:
            c.implicit_setup(1.0, 1e-2)
    r, phi, z = g.nodes3()
    if kind == B.NONLIN_VORTEX:
        s0 = np.concatenate([W.random_spectral(g.nc, g.M, g.Kz, seed=4, scale_decay=0.5),
                             W.random_spectral(g.nc, g.M, g.Kz, seed=5, scale_decay=0.5)]) * 1e-2
    else:
        s0 = O.to_flat(g, O.forward(g, W.fkpp_seed(r, phi, z)))
    coeff = [1.0]
    full = to_gpu_spec(s0)
    pf = torch.zeros_like(full)
    a_ctx.advance(kind, coeff, full, pf, 10, True)
    part = to_gpu_spec(s0)
    pp = torch.zeros_like(part)
    a_ctx.advance(kind, coeff, part, pp, 4, True)
    img = a_ctx.get_state(kind, part, pp, step=4)
    assert len(img) == a_ctx.state_bytes(kind) > 2 * nf * a_ctx.n_spec * 16
    rs, rp = torch.zeros_like(part), torch.zeros_like(part)
    assert b_ctx.set_state(kind, img, rs, rp) == 4
    b_ctx.advance(kind, coeff, rs, rp, 6, False)
    assert np.array_equal(rs.cpu().numpy(), full.cpu().numpy())
    assert np.array_equal(rp.cpu().numpy(), pf.cpu().numpy())
    # another time step (or another grid) cannot continue the AB-CN recurrence
    _, c_ctx = pair(nr, nphi, nz, ell, lz=lz, policy="twothirds")
    if kind == B.NONLIN_VORTEX:
        c_ctx.vortex_setup()
        c_ctx.implicit_setup(1e-3, 2e-3, nu_h=5e-7, p=8)
    else:
        c_ctx.implicit_setup(1.0, 2e-2)
    with pytest.raises(B.MlxError) as e:
        c_ctx.set_state(kind, img, rs, rp)
    assert e.value.code == -1
    _, d_ctx = pair(nr + 1, nphi, nz, ell, lz=lz, policy="twothirds")
    with pytest.raises(B.MlxError):
        d_ctx.set_state(kind, img, torch.zeros(len(img) // 16, dtype=torch.complex128, device="cuda"),
                        torch.zeros(len(img) // 16, dtype=torch.complex128, device="cuda"))


@pytest.mark.parametrize("prec", [B.FP64, B.FP32, B.BF16X3])
@pytest.mark.parametrize("kind", [B.NONLIN_FKPP, B.NONLIN_VORTEX])
def test_nonfinite_state_sets_enumeric(kind, prec):
    # a NaN planted in the state on the host: the nonlinear kernels flag the
    # non-finite product, mlx_device_status returns MLX_ENUMERIC once and clears it;
    # a clean call afterwards leaves the word clear
    g, ctx = pair(24, 16, 8, 1.0, lz=8.6, policy="twothirds", precision=prec)
    nf = 1
    if kind == B.NONLIN_VORTEX:
        ctx.vortex_setup()
        nf = 2
    good = np.concatenate([W.random_spectral(g.nc, g.M, g.Kz, seed=7 + f, scale_decay=0.5) for f in range(nf)])
    bad = good.copy()
    bad[3] = np.nan
    out = to_gpu_spec(np.zeros_like(good))
    ctx.device_status()
    ctx.nonlinear(kind, [1.0], to_gpu_spec(bad), out)
    with pytest.raises(B.MlxError) as e:
        ctx.device_status()
    assert e.value.code == -3
    ctx.device_status()                     # cleared by the read
    ctx.nonlinear(kind, [1.0], to_gpu_spec(good), out)
    ctx.device_status()
