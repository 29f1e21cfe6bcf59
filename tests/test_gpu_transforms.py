"""GPU parity of nodes, transforms and the nonlinear term against the oracle.

Bars: FP64 form within 1e-12 relative (spectral l2 with multiplicity 2 for
m >= 1, or l2 over the nodes); FP32 form within 1e-6 relative.
"""

import numpy as np
import pytest

import oracle as O
from paper_2609_18026_b300 import binding as B

from gpu_common import (pair, to_gpu_phys, to_gpu_spec, spec_from_gpu, rand_phys, rand_spec, rel,
                        block_err, max_err)

pytestmark = pytest.mark.gpu

GRIDS = [
    # nr, nphi, nz, ell, policy       (tiny, ragged, several tiles, Nz = 1 and > 1)
    (4, 4, 1, 1.0, "linear"),
    (5, 8, 4, 0.8, "linear"),
    (33, 16, 8, 1.7, "twothirds"),
    (70, 32, 16, 2.0, "linear"),
    (100, 64, 1, 4.0, "twothirds"),
    (128, 128, 64, 4.0, "twothirds"),
    (9, 256, 32, 1.0, "linear", 7),       # in-lane butterfly stages (E = 8), M = 7
    (6, 512, 2, 1.0, "twothirds", 5),     # E = 16, Nz = 2, M = 5
    (12, 4, 256, 0.7, "linear"),          # lane groups for Nphi = 4, long z lines
    # Nyquist-keeping chop (|m| <= Nphi/2, |k| <= Nz/2): the pair splitting of the
    # forward direction and the pair sums of the backward one
    (9, 8, 2, 1.0, "nyquist"),            # Nz = 2: K = 3, both k = +-1 rows are the pair
    (24, 16, 8, 1.3, "nyquist"),
    (70, 32, 16, 2.0, "nyquist"),
    (40, 64, 1, 2.0, "nyquist"),          # 2-D: azimuthal pair only
    (12, 4, 256, 0.7, "nyquist"),         # M = 3 with Nphi = 4, K = 257
    (256, 256, 32, 4.0, "nyquist"),       # M = 129: the production run's azimuthal chop
]
TOL = {B.FP64: 1e-12, B.FP32: 1e-6, B.BF16X3: 1e-6}
# element-wise bars: every (m, k) block of a spectral result (or every node of a
# physical one) within BLOCK times that block's own largest value; for smooth
# inputs whose spectra decay, blocks below FLOOR of the largest block are held
# to FLOOR times it (the transforms' rounding is absolute, at the global scale)
BLOCK = {B.FP64: 1e-11, B.FP32: 1e-5, B.BF16X3: 1e-5}
FLOOR = {B.FP64: 1e-3, B.FP32: 0.1, B.BF16X3: 0.1}
PNAME = {B.FP64: "fp64", B.FP32: "fp32", B.BF16X3: "bf16x3"}
PRECS = [B.FP64, B.FP32, B.BF16X3]


@pytest.mark.parametrize("nr", [2, 24, 96, 256, 1024])
def test_nodes_weights_radii(nr):
    g, ctx = pair(nr, 4, 1, 1.3)
    x, w, r = ctx.nodes()
    assert np.max(np.abs(x - g.x)) <= 4e-16
    assert np.max(np.abs(w - g.w) / g.w) <= 1e-12
    assert np.max(np.abs(r - g.r) / g.r) <= 1e-12


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("grid", GRIDS)
def test_forward_parity(grid, prec, record):
    nr, nphi, nz, ell, pol = grid[:5]
    chop = dict(nphi_c=grid[5]) if len(grid) > 5 else {}
    g, ctx = pair(nr, nphi, nz, ell, lz=3.7, policy=pol, precision=prec, **chop)
    f = rand_phys(g, 11)
    if prec != B.FP64:
        f = f.astype(np.float32).astype(np.float64)   # both sides see the same input
    spec = ctx.forward(to_gpu_phys(ctx, f), ctx.new_spec())
    got = spec_from_gpu(g, spec)
    ref = O.forward(g, f)
    e, eb = O.spec_rel_err(g, got, ref), block_err(g, got, ref)
    record("forward", grid=grid[:3], precision=PNAME[prec], rel_err=e, block_err=eb)
    assert e <= TOL[prec]
    assert eb <= BLOCK[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("grid", GRIDS)
def test_backward_parity(grid, prec, record):
    nr, nphi, nz, ell, pol = grid[:5]
    chop = dict(nphi_c=grid[5]) if len(grid) > 5 else {}
    g, ctx = pair(nr, nphi, nz, ell, lz=3.7, policy=pol, precision=prec, **chop)
    flat = rand_spec(g, 5)
    phys = ctx.backward(to_gpu_spec(flat), ctx.new_phys())
    got = phys.double().cpu().numpy()
    ref = O.backward(g, O.from_flat(g, flat))
    e, em = rel(got, ref), max_err(got, ref)
    record("backward", grid=grid[:3], precision=PNAME[prec], rel_err=e, max_err=em)
    assert e <= TOL[prec]
    assert em <= BLOCK[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_roundtrip_identity(prec):
    g, ctx = pair(64, 32, 16, 1.0, policy="twothirds", precision=prec)
    flat = rand_spec(g, 9)
    s = to_gpu_spec(flat)
    back = ctx.forward(ctx.backward(s, ctx.new_phys()), ctx.new_spec())
    # two transforms in sequence, each within TOL: the composition is within 2 TOL
    assert O.spec_rel_err(g, spec_from_gpu(g, back), O.from_flat(g, flat)) <= 2 * TOL[prec]


def test_azimuthal_purity_exact():
    # Sec. 5.1: odd harmonics of a cos(2 phi) field are identically zero.  The
    # input is made bitwise periodic under phi -> phi + pi; the FFT's first
    # butterfly then cancels exactly.
    g, ctx = pair(48, 16, 1, 1.0)
    r, phi, z = g.nodes3()
    j = np.arange(g.nphi)
    c2 = np.cos(2 * np.pi * ((2 * j) % g.nphi) / g.nphi)
    f = (r ** 2 * np.exp(-r ** 2 / 2)) * c2[None, :, None] + 0 * z
    spec = spec_from_gpu(g, ctx.forward(to_gpu_phys(ctx, f), ctx.new_spec()))
    for m in range(1, g.M, 2):
        assert np.all(spec[m] == 0.0)
    assert np.max(np.abs(spec[0])) < 1e-16


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("grid", [(5, 8, 4, 0.8), (40, 16, 8, 2.0), (128, 128, 64, 4.0),
                                  (40, 16, 8, 2.0, "nyquist"), (64, 32, 1, 2.0, "nyquist")])
def test_fkpp_nonlinear_parity(grid, prec, record):
    nr, nphi, nz, ell = grid[:4]
    pol = grid[4] if len(grid) > 4 else "twothirds"
    g, ctx = pair(nr, nphi, nz, ell, lz=2 * np.pi * 8, policy=pol, precision=prec)
    r, phi, z = g.nodes3()
    from paper_2609_18026_b300 import workloads as W
    s0 = O.forward(g, W.fkpp_seed(r, phi, z))
    out = ctx.nonlinear(B.NONLIN_FKPP, [1.0], to_gpu_spec(O.to_flat(g, s0)), ctx.new_spec())
    ref = O.fkpp_nonlinear(g, 1.0)(s0)
    got = spec_from_gpu(g, out)
    e, eb = O.spec_rel_err(g, got, ref), block_err(g, got, ref, floor=FLOOR[prec])
    record("fkpp_nonlinear", grid=grid[:3], policy=pol, precision=PNAME[prec], rel_err=e, block_err=eb)
    assert e <= TOL[prec]
    assert eb <= BLOCK[prec]


@pytest.mark.parametrize("grid", [(256, 256, 16, 1.0), (256, 64, 64, 2.0), (200, 32, 8, 1.0)])
def test_tc_contraction_nr256(grid, record):
    # the tensor-core contraction at the vortex workload's radial size (Nr = Nc =
    # 256: two 128-lane row tiles, four 64-wide K chunks per tile; M = 86 at
    # Nphi = 256) and at a ragged Nr = 200, both directions, against the oracle
    nr, nphi, nz, ell = grid
    g, ctx = pair(nr, nphi, nz, ell, lz=8.6, policy="twothirds", precision=B.BF16X3)
    flat = rand_spec(g, 6)
    phys = ctx.backward(to_gpu_spec(flat), ctx.new_phys()).double().cpu().numpy()
    ref = O.backward(g, O.from_flat(g, flat))
    eb, emb = rel(phys, ref), max_err(phys, ref)
    u = rand_phys(g, 7).astype(np.float32).astype(np.float64)
    spec = spec_from_gpu(g, ctx.forward(to_gpu_phys(ctx, u), ctx.new_spec()))
    reff = O.forward(g, u)
    ef, efb = O.spec_rel_err(g, spec, reff), block_err(g, spec, reff)
    record("tc_nr256", grid=grid, backward_rel=eb, backward_max=emb, forward_rel=ef, forward_block=efb)
    assert eb <= 1e-6 and emb <= 1e-5
    assert ef <= 1e-6 and efb <= 1e-5
    ctx.device_status()


@pytest.mark.parametrize("tile", [2, 4, 16])
def test_fft_tile_sizes_agree(tile):
    # the phi kernel pairs radii r and r + tile/2 into one complex line, the z
    # kernel transforms tile radii per CTA: other tiles, same transforms (odd Nr)
    g, ctx = pair(33, 16, 8, 1.7, lz=2 * np.pi * 8, policy="twothirds", precision=B.FP32)
    r, phi, z = g.nodes3()
    from paper_2609_18026_b300 import workloads as W
    s0 = to_gpu_spec(O.to_flat(g, O.forward(g, W.fkpp_seed(r, phi, z))))
    outs = []
    for t in (32, tile):
        ctx.set_tuning("phi_tile", t)
        ctx.set_tuning("z_tile", t)
        outs.append(ctx.nonlinear(B.NONLIN_FKPP, [1.0], s0, ctx.new_spec()).cpu().numpy())
        outs.append(ctx.forward(ctx.backward(s0, ctx.new_phys()), ctx.new_spec()).cpu().numpy())
    for a, b in ((outs[0], outs[2]), (outs[1], outs[3])):
        assert np.linalg.norm(b - a) <= 1e-6 * np.linalg.norm(a)


@pytest.mark.parametrize("bn", [16, 48])
def test_tc_column_tile_widths(bn):
    # the tensor-core contraction at other column-tile widths (N = 16 is the
    # smallest MMA width at M = 128) against the oracle, both directions
    g, ctx = pair(128, 128, 64, 4.0, policy="twothirds", precision=B.BF16X3)
    ctx.set_tuning("tc_bn", bn)
    flat = rand_spec(g, 4)
    phys = ctx.backward(to_gpu_spec(flat), ctx.new_phys())
    ref = O.backward(g, O.from_flat(g, flat))
    assert rel(phys.double().cpu().numpy(), ref) <= 1e-6
    u = rand_phys(g, 5)
    spec = ctx.forward(to_gpu_phys(ctx, u), ctx.new_spec())
    assert O.spec_rel_err(g, spec_from_gpu(g, spec), O.forward(g, u.astype(np.float32).astype(np.float64))) <= 1e-6
    ctx.device_status()


def test_bf16x3_device_status_clean():
    # the tensor-core kernels' bounded waits never expire on a normal run
    g, ctx = pair(128, 128, 64, 4.0, policy="twothirds", precision=B.BF16X3)
    flat = rand_spec(g, 4)
    ctx.forward(ctx.backward(to_gpu_spec(flat), ctx.new_phys()), ctx.new_spec())
    ctx.device_status()


@pytest.mark.parametrize("direction", ["forward", "backward"])
def test_tc_forced_wait_expiry_reports_timeout(direction):
    # The tensor-core contraction's bounded waits: with the test hook "tc_expire"
    # the first shared-memory stage-reuse wait reports expiry at once; the kernel
    # must drain what it issued, free its tensor memory and return, the context
    # must report MLX_ETIMEOUT once, and the next normal call must be clean and
    # correct.  Nr = 256 gives 6-8 K chunks per work item (more than the 4 stages).
    g, ctx = pair(256, 64, 16, 1.0, lz=8.6, policy="twothirds", precision=B.BF16X3)
    u = rand_phys(g, 7).astype(np.float32).astype(np.float64)
    flat = rand_spec(g, 6)

    def run():
        if direction == "forward":
            return ctx.forward(to_gpu_phys(ctx, u), ctx.new_spec())
        return ctx.backward(to_gpu_spec(flat), ctx.new_phys())
    ctx.device_status()
    ctx.set_tuning("tc_expire", 1)
    run()
    with pytest.raises(B.MlxError) as e:
        ctx.device_status()
    assert e.value.code == -4
    ctx.set_tuning("tc_expire", 0)
    out = run()
    ctx.device_status()
    if direction == "forward":
        assert O.spec_rel_err(g, spec_from_gpu(g, out), O.forward(g, u)) <= 1e-6
    else:
        assert rel(out.double().cpu().numpy(), O.backward(g, O.from_flat(g, flat))) <= 1e-6
