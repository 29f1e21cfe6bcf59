"""GPU parity of the adaptive modal filter (Sec. 3.3) against the oracle."""

import numpy as np
import pytest

import oracle as O
from oracle import filter as F
from paper_2609_18026_b300 import binding as B
from paper_2609_18026_b300 import workloads as W

from gpu_common import pair, to_gpu_spec, spec_from_gpu, block_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("decay", [0.0, 0.6])
def test_filter_apply_parity(decay, record):
    # three consecutive filter steps on one field: the white spectrum drives eps up
    # its relaxation ramp, the decaying one keeps it lower; coefficients element by
    # element and the amplitude against the oracle
    g, ctx = pair(40, 16, 8, 1.5, lz=3.0, policy="twothirds")
    ctx.filter_setup(True)
    flat = W.random_spectral(g.nc, g.M, g.Kz, seed=8, scale_decay=decay)
    dev = to_gpu_spec(flat)
    ref, eps = O.from_flat(g, flat), 0.0
    for step in range(3):
        ctx.filter_apply(dev, 1)
        ref, eps, f = F.apply(g, ref, eps)
        ge, gt = ctx.filter_state()
        got = spec_from_gpu(g, dev)
        e, eb = O.spec_rel_err(g, got, ref), block_err(g, got, ref, floor=1e-12)
        record("filter_apply", decay=decay, step=step, eps=eps, tail=f, rel_err=e, block_err=eb)
        assert abs(ge[0] - eps) <= 1e-12 * max(1.0, eps)
        assert abs(gt[0] - f) <= 1e-13
        assert e <= 1e-13 and eb <= 1e-12


@pytest.mark.parametrize("kind,prec,tol", [(B.NONLIN_FKPP, B.FP64, 1e-12), (B.NONLIN_FKPP, B.BF16X3, 1e-6),
                                           (B.NONLIN_VORTEX, B.FP64, 1e-12)])
def test_advance_with_filter_parity(kind, prec, tol, record):
    # the filter between steps inside the graph-replayed advance: every field has its
    # own amplitude; against the oracle stepper with the same filter after every step
    nr, nphi, nz, ell, lz = 24, 16, 8, 1.0, 8.6
    g, ctx = pair(nr, nphi, nz, ell, lz=lz, policy="twothirds", precision=prec)
    nf = 2 if kind == B.NONLIN_VORTEX else 1
    if kind == B.NONLIN_VORTEX:
        ctx.vortex_setup()
        ctx.implicit_setup(1e-3, 1e-3, nu_h=5e-7, p=8)
        s0 = np.concatenate([W.random_spectral(g.nc, g.M, g.Kz, seed=9 + f, scale_decay=0.3) * 1e-2
                             for f in range(2)])
        A, _ = O.vortex_nonlinear(g, 1.0, form="banded")
        st = O.Stepper(g, 1e-3, 1e-3, nu_h=5e-7, p=8, nonlinear=A, post=F.FieldFilter(g, 2))
    else:
        ctx.implicit_setup(1.0, 1e-2)
        s0 = W.random_spectral(g.nc, g.M, g.Kz, seed=9, scale_decay=0.1) * 1e-2
        st = O.Stepper(g, 1.0, 1e-2, nonlinear=O.fkpp_nonlinear(g, 1.0), post=F.FieldFilter(g, 1))
    ctx.filter_setup(True)
    state = to_gpu_spec(s0)
    prev = to_gpu_spec(np.zeros_like(s0))
    ctx.advance(kind, [1.0], state, prev, 7, True)
    n = len(s0) // nf
    blocks = [O.from_flat(g, s0[f * n:(f + 1) * n]) for f in range(nf)]
    ref, _ = st.run_abcn(sum(blocks, []), 7)
    o = state.cpu().numpy()
    got = sum([O.from_flat(g, o[f * n:(f + 1) * n]) for f in range(nf)], [])
    e = O.spec_rel_err(g, got, ref)
    geps, _ = ctx.filter_state()
    record("advance_filter", kind=kind, precision=prec, rel_err=e, eps=geps[:nf], eps_oracle=st.post.eps)
    assert e <= tol
    for f in range(nf):
        assert abs(geps[f] - st.post.eps[f]) <= max(1e-10, 1e-4 * tol * 1e6) * max(1.0, st.post.eps[f])
    assert max(st.post.eps) > 0.0             # the filter acted
    ctx.device_status()
