"""Batched uneven solves (one CUDA graph per step pair) and the autotuner."""

import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2609_18026_b300 import binding as B
from paper_2609_18026_b300 import workloads as W

from gpu_common import spec_from_gpu, block_err

pytestmark = pytest.mark.gpu

# uneven instances: (nr, nphi, nz, ell, kind, precision)
INST = [(32, 16, 1, 0.7, B.NONLIN_NONE, B.FP32),
        (48, 32, 16, 2.0, B.NONLIN_FKPP, B.FP32),
        (64, 16, 16, 3.1, B.NONLIN_FKPP, B.BF16X3),
        (40, 64, 1, 1.3, B.NONLIN_NONE, B.BF16X3),
        (24, 8, 4, 0.9, B.NONLIN_FKPP, B.FP64)]


def _make(inst, seed):
    import torch
    nr, nphi, nz, ell, kind, prec = inst
    ctx = B.Context(nr, nphi, nz, ell, lz=2 * math.pi, precision=prec, chop_policy=B.CHOP_LINEAR)
    ctx.implicit_setup(1e-2 if kind == B.NONLIN_NONE else 1.0, 1e-3)
    x, w, r = ctx.nodes()
    phi = 2 * np.pi * np.arange(nphi) / nphi
    zz = 2 * np.pi * np.arange(nz) / nz
    par = dict(x0=0.3 * ell, y0=-0.2 * ell, sigma=ell, nz=nz, lz=2 * math.pi)
    u0 = W.batch_initial(par, r[None, None, :], phi[None, :, None], zz[:, None, None])
    s = ctx.forward(torch.as_tensor(u0, dtype=ctx.phys_dtype).cuda(), ctx.new_spec())
    return ctx, s, u0


@pytest.mark.parametrize("persistent", [1, 0])
def test_batched_advance_equals_individual(persistent):
    # persistent: every phase one queue launch over all members (tensor-core,
    # FP32 and FP64 SIMT contractions, 2-D and 3-D FFT stages, solves with and
    # without a nonlinear term); 0: one graph branch per member
    ctxs, s_b, s_i, p_b, p_i = [], [], [], [], []
    for j, inst in enumerate(INST):
        ctx, s, _ = _make(inst, j)
        ctxs.append(ctx)
        s_b.append(s.clone()); s_i.append(s.clone())
        p_b.append(ctx.new_spec()); p_i.append(ctx.new_spec())
    kinds = [inst[4] for inst in INST]
    coeffs = [1.0] * len(INST)
    batch = B.Batch(ctxs)
    batch.set_persistent(persistent)
    batch.advance(kinds, coeffs, s_b, p_b, 7, True)
    batch.advance(kinds, coeffs, s_b, p_b, 6, False)
    for j, ctx in enumerate(ctxs):
        ctx.advance(kinds[j], [1.0], s_i[j], p_i[j], 7, True)
        ctx.advance(kinds[j], [1.0], s_i[j], p_i[j], 6, False)
    for j in range(len(INST)):
        assert np.array_equal(s_b[j].cpu().numpy(), s_i[j].cpu().numpy()), j
        assert np.array_equal(p_b[j].cpu().numpy(), p_i[j].cpu().numpy()), j
    batch.close()


def test_batched_instance_matches_oracle():
    inst = INST[1]
    ctx, s, u0 = _make(inst, 1)
    batch = B.Batch([ctx])
    p = ctx.new_spec()
    batch.advance([inst[4]], [1.0], [s], [p], 5, True)
    nr, nphi, nz, ell, kind, prec = inst
    g = O.Grid(nr, nphi, nz, ell, lz=2 * math.pi, policy="linear")
    u0 = u0.astype(np.float32).astype(np.float64)
    st = O.Stepper(g, 1.0, 1e-3, nonlinear=O.fkpp_nonlinear(g, 1.0))
    ref, _ = st.run_abcn(O.forward(g, u0), 5)
    assert O.spec_rel_err(g, spec_from_gpu(g, s), ref) <= 1e-6


def test_autotune_cache_roundtrip(tmp_path):
    import torch
    cache = str(tmp_path / "tune.txt")
    inst = (128, 128, 64, 4.0, B.NONLIN_FKPP, B.BF16X3)
    ctx = B.Context(128, 128, 64, 4.0, lz=2 * np.pi * 8, precision=B.BF16X3, chop_policy=B.CHOP_TWOTHIRDS)
    ctx.implicit_setup(1.0, 1e-2)
    first = ctx.autotune(B.NONLIN_FKPP, [1.0], cache)
    assert not first["from_cache"]
    # cpw = 0 denotes the segmented solve, cpw = 2 the lean variant (wpb = 0 for both)
    assert first["cpw"] in (0, 2, 4, 8, 16, 32) and first["wpb"] in (0, 1, 2, 4) and 16 <= first["bn"] <= 256
    assert os.path.exists(cache)
    ctx2 = B.Context(128, 128, 64, 4.0, lz=2 * np.pi * 8, precision=B.BF16X3, chop_policy=B.CHOP_TWOTHIRDS)
    ctx2.implicit_setup(1.0, 1e-2)
    second = ctx2.autotune(B.NONLIN_FKPP, [1.0], cache)
    assert second["from_cache"] and second == dict(first, from_cache=True)
    # the tuned shapes change the arithmetic order only: results agree to 1e-6
    g = O.Grid(128, 128, 64, 4.0, lz=2 * np.pi * 8, policy="twothirds")
    r, phi, z = g.nodes3()
    u0 = W.fkpp_seed(r, phi, z).astype(np.float32)
    ref_ctx = B.Context(128, 128, 64, 4.0, lz=2 * np.pi * 8, precision=B.BF16X3, chop_policy=B.CHOP_TWOTHIRDS)
    ref_ctx.implicit_setup(1.0, 1e-2)
    outs = []
    for c in (ctx2, ref_ctx):
        s = c.forward(torch.as_tensor(u0).cuda(), c.new_spec())
        p = c.new_spec()
        c.advance(B.NONLIN_FKPP, [1.0], s, p, 10, True)
        outs.append(O.from_flat(g, s.cpu().numpy()))
    assert O.spec_rel_err(g, outs[0], outs[1]) <= 1e-6


def test_batch64_every_instance_matches_oracle(record):
    # The benchmarked 64-instance uneven batch (seed 20261202: Nr in {32..256},
    # Nphi in {16..256}, Nz in {1, 16, 64}, ell in [0.5, 4], diffusion or
    # Fisher-KPP), built exactly as the benchmark builds it (BF16x3 contraction,
    # FP32 FFTs, FP64 solves, dt = 1e-3), advanced 3 steps (Richardson start +
    # 2 AB-CN) through one batch graph from the oracle's FP64 initial
    # coefficients: every instance against the oracle, globally and per block.
    import torch
    insts = W.batch_instances(64)
    ctxs, states, prevs, kinds, grids, s0s, steppers = [], [], [], [], [], [], []
    for inst in insts:
        lin = inst["kind"] == "diffusion"
        pol = B.CHOP_LINEAR if lin else B.CHOP_TWOTHIRDS
        m_pol = inst["nphi"] // 2 if lin else (inst["nphi"] - 1) // 3 + 1
        M = min(m_pol, inst["nr"])
        ctx = B.Context(inst["nr"], inst["nphi"], inst["nz"], inst["ell"], lz=inst["lz"], precision=B.BF16X3,
                        chop_policy=pol, nphi_c=M)
        kind = B.NONLIN_NONE if lin else B.NONLIN_FKPP
        nu = 1e-2 if lin else 1.0
        ctx.implicit_setup(nu, inst["dt"])
        g = O.Grid(inst["nr"], inst["nphi"], inst["nz"], inst["ell"], lz=inst["lz"],
                   policy="linear" if lin else "twothirds", M=M)
        r, phi, z = g.nodes3()
        s0 = O.forward(g, W.batch_initial(inst, r, phi, z))
        ctxs.append(ctx); kinds.append(kind); grids.append(g); s0s.append(s0)
        states.append(torch.as_tensor(O.to_flat(g, s0)).cuda()); prevs.append(ctx.new_spec())
        steppers.append(O.Stepper(g, nu, inst["dt"], nonlinear=None if lin else O.fkpp_nonlinear(g, 1.0)))
    batch = B.Batch(ctxs)
    batch.advance(kinds, [1.0] * 64, states, prevs, 3, True)
    torch.cuda.synchronize()
    worst, worst_blk = 0.0, 0.0
    for j in range(64):
        ref, _ = steppers[j].run_abcn(s0s[j], 3)
        got = spec_from_gpu(grids[j], states[j])
        e = O.spec_rel_err(grids[j], got, ref)
        eb = block_err(grids[j], got, ref, floor=0.1)
        worst, worst_blk = max(worst, e), max(worst_blk, eb)
        assert e <= 1e-6, (j, insts[j], e)
        assert eb <= 1e-5, (j, insts[j], eb)
    record("batch64_vs_oracle", worst_rel_err=worst, worst_block_err=worst_blk)
    batch.close()


def test_batch64_persistent_equals_branches():
    # The 64-instance uneven workload: the per-phase persistent launches (one
    # tensor-core launch over all 33 BF16x3 Fisher-KPP members, queue-fed FFT
    # stages and solves) against one graph branch per member, bitwise, over a
    # Richardson start and 6 AB-CN steps (3 replayed pairs).
    import torch
    insts = W.batch_instances(64)
    ctxs, kinds, s0 = [], [], []
    for inst in insts:
        lin = inst["kind"] == "diffusion"
        pol = B.CHOP_LINEAR if lin else B.CHOP_TWOTHIRDS
        m_pol = inst["nphi"] // 2 if lin else (inst["nphi"] - 1) // 3 + 1
        ctx = B.Context(inst["nr"], inst["nphi"], inst["nz"], inst["ell"], lz=inst["lz"], precision=B.BF16X3,
                        chop_policy=pol, nphi_c=min(m_pol, inst["nr"]))
        kind = B.NONLIN_NONE if lin else B.NONLIN_FKPP
        ctx.implicit_setup(1e-2 if lin else 1.0, inst["dt"])
        x, w, r = ctx.nodes()
        phi = 2 * np.pi * np.arange(inst["nphi"]) / inst["nphi"]
        zz = inst["lz"] * np.arange(inst["nz"]) / inst["nz"]
        u0 = W.batch_initial(inst, r[None, None, :], phi[None, :, None], zz[:, None, None])
        s0.append(ctx.forward(torch.as_tensor(u0, dtype=torch.float32).cuda(), ctx.new_spec()))
        ctxs.append(ctx); kinds.append(kind)
    batch = B.Batch(ctxs)
    out = []
    for mode in (1, 0):
        batch.set_persistent(mode)
        st = [s.clone() for s in s0]
        pv = [c.new_spec() for c in ctxs]
        batch.advance(kinds, [1.0] * 64, st, pv, 7, True)
        torch.cuda.synchronize()
        out.append(([s.cpu().numpy() for s in st], [p.cpu().numpy() for p in pv]))
    for j in range(64):
        assert np.isfinite(out[0][0][j]).all(), j
        assert np.array_equal(out[0][0][j], out[1][0][j]), (j, insts[j])
        assert np.array_equal(out[0][1][j], out[1][1][j]), (j, insts[j])
    for c in ctxs:
        c.device_status()   # raises on an expired bounded wait or a non-finite product
    batch.close()


def test_batch_tensor_core_launches_split_past_64_members():
    # 70 small BF16x3 Fisher-KPP members: the tensor-core contraction takes at most
    # 64 members' maps per launch, so each direction runs as two launches; the
    # persistent graph still matches the per-member branches bitwise.
    import torch
    ctxs, s0 = [], []
    rng = np.random.default_rng(70)
    for j in range(70):
        nr = int(rng.choice([16, 24, 32]))
        nphi = int(rng.choice([8, 16]))
        nz = int(rng.choice([1, 4]))
        ell = float(rng.uniform(0.7, 2.0))
        ctx = B.Context(nr, nphi, nz, ell, lz=2 * math.pi, precision=B.BF16X3, chop_policy=B.CHOP_TWOTHIRDS)
        ctx.implicit_setup(1.0, 1e-3)
        x, w, r = ctx.nodes()
        phi = 2 * np.pi * np.arange(nphi) / nphi
        zz = 2 * np.pi * np.arange(nz) / nz
        par = dict(x0=0.2 * ell, y0=0.1 * ell, sigma=ell, nz=nz, lz=2 * math.pi)
        u0 = W.batch_initial(par, r[None, None, :], phi[None, :, None], zz[:, None, None])
        s0.append(ctx.forward(torch.as_tensor(u0, dtype=torch.float32).cuda(), ctx.new_spec()))
        ctxs.append(ctx)
    kinds = [B.NONLIN_FKPP] * 70
    batch = B.Batch(ctxs)
    out = []
    for mode in (1, 0):
        batch.set_persistent(mode)
        st = [s.clone() for s in s0]
        pv = [c.new_spec() for c in ctxs]
        batch.advance(kinds, [1.0] * 70, st, pv, 5, True)
        torch.cuda.synchronize()
        out.append([s.cpu().numpy() for s in st])
    for j in range(70):
        assert np.isfinite(out[0][j]).all(), j
        assert np.array_equal(out[0][j], out[1][j]), j
    for c in ctxs:
        c.device_status()
    batch.close()
