"""GPU parity of the FP64 banded implicit solve and of the time advance."""

import numpy as np
import pytest

import oracle as O
from paper_2609_18026_b300 import binding as B
from paper_2609_18026_b300 import workloads as W

from gpu_common import pair, to_gpu_spec, spec_from_gpu, rand_spec

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("pol", ["twothirds", "nyquist"])
@pytest.mark.parametrize("nu_h,p", [(0.0, 8), (5e-3, 4), (5e-7, 8)])
@pytest.mark.parametrize("step", [B.STEP_FEBE_HALF, B.STEP_FEBE_FULL, B.STEP_ABCN])
def test_implicit_solve_parity(step, nu_h, p, pol):
    g, ctx = pair(40, 16, 8, 1.5, lz=3.0, policy=pol)
    dt, nu = 2e-2, 0.3
    ctx.implicit_setup(nu, dt, nu_h=nu_h, p=p)
    st = O.Stepper(g, nu, dt, nu_h=nu_h, p=p)
    s = rand_spec(g, 1)
    A = rand_spec(g, 2)
    Ap = rand_spec(g, 3)
    out = ctx.implicit_solve(step, to_gpu_spec(s), to_gpu_spec(A), to_gpu_spec(Ap), ctx.new_spec())
    S, AA, AP = (O.from_flat(g, v) for v in (s, A, Ap))
    if step == B.STEP_ABCN:
        ref = st.abcn(S, AA, AP)
    else:
        ref = st.febe(S, step == B.STEP_FEBE_HALF, AA)
    # Bar: 1e-12, or the FP64 perturbation bound 2 kappa u of a backward-stable
    # solve when the systems are worse conditioned than 1e12 * u allows (the p = 8
    # hyperviscous operator reaches kappa ~ 1e5 here; the oracle itself is 1.5e-12
    # from a 50-digit solve on those systems).
    c = 0.5 * dt if step != B.STEP_FEBE_FULL else dt
    kappa = max(np.linalg.cond(np.eye(L.shape[0]) - c * L) for L in st.L.values())
    tol = max(1e-12, 2.0 * kappa * 2.0 ** -53)
    assert O.spec_rel_err(g, spec_from_gpu(g, out), ref) <= tol


@pytest.mark.parametrize("step", [B.STEP_FEBE_HALF, B.STEP_ABCN])
def test_implicit_solve_parity_smooth_rhs(step):
    # Spectrally decaying right-hand sides (what the time loop sees): 1e-12 even
    # with the p = 8 hyperviscous operator.
    g, ctx = pair(40, 16, 8, 1.5, lz=3.0, policy="twothirds")
    dt, nu = 2e-2, 0.3
    ctx.implicit_setup(nu, dt, nu_h=5e-7, p=8)
    st = O.Stepper(g, nu, dt, nu_h=5e-7, p=8)
    s, A, Ap = (rand_spec(g, k) for k in (1, 2, 3))
    S, AA, AP = (O.from_flat(g, v) for v in (s, A, Ap))
    for blk in (S, AA, AP):
        for m, b in enumerate(blk):
            b *= np.exp(-0.3 * np.arange(m, g.nc))[None, :]
    out = ctx.implicit_solve(step, *(to_gpu_spec(O.to_flat(g, v)) for v in (S, AA, AP)), ctx.new_spec())
    ref = st.abcn(S, AA, AP) if step == B.STEP_ABCN else st.febe(S, True, AA)
    assert O.spec_rel_err(g, spec_from_gpu(g, out), ref) <= 1e-12


def test_solve_before_setup_is_state_error():
    g, ctx = pair(8, 8, 1, 1.0)
    s = to_gpu_spec(rand_spec(g, 1))
    with pytest.raises(B.MlxError) as e:
        ctx.implicit_solve(B.STEP_ABCN, s, None, None, ctx.new_spec())
    assert e.value.code == -5


def test_polar_diffusion_100_steps():
    # 2-D polar diffusion, Nr = Nphi = 32, ell = 1, nu = 1e-2, dt = 1e-3, 100 AB-CN
    # steps (Richardson start), exp(-r^2)(1 + 0.5 cos 2 phi): FP64 parity.
    g, ctx = pair(32, 32, 1, 1.0)
    r, phi, z = g.nodes3()
    s0 = O.forward(g, W.gaussian_polar(r, phi, z))
    ctx.implicit_setup(1e-2, 1e-3)
    state = to_gpu_spec(O.to_flat(g, s0))
    prevA = ctx.new_spec()
    ctx.advance(B.NONLIN_NONE, [], state, prevA, 100, True)
    ref, _ = O.Stepper(g, 1e-2, 1e-3).run_abcn(s0, 100)
    assert O.spec_rel_err(g, spec_from_gpu(g, state), ref) <= 1e-12


@pytest.mark.parametrize("pol", ["twothirds", "nyquist"])
@pytest.mark.parametrize("prec,tol", [(B.FP64, 1e-12), (B.FP32, 1e-6), (B.BF16X3, 1e-6)])
def test_fkpp_advance_small(prec, tol, pol):
    g, ctx = pair(24, 16, 8, 4.0, lz=2 * np.pi * 8, policy=pol, precision=prec)
    r, phi, z = g.nodes3()
    s0 = O.forward(g, W.fkpp_seed(r, phi, z))
    dt = 1e-2
    ctx.implicit_setup(1.0, dt)
    state = to_gpu_spec(O.to_flat(g, s0))
    prevA = ctx.new_spec()
    # split into two calls (odd then even) to cover the resume path
    ctx.advance(B.NONLIN_FKPP, [1.0], state, prevA, 7, True)
    ctx.advance(B.NONLIN_FKPP, [1.0], state, prevA, 6, False)
    ref, _ = O.Stepper(g, 1.0, dt, nonlinear=O.fkpp_nonlinear(g, 1.0)).run_abcn(s0, 13)
    assert O.spec_rel_err(g, spec_from_gpu(g, state), ref) <= tol


def test_advance_checkpoint_resume_bitwise():
    # N steps == k steps + save/load + (N - k) steps, bitwise in FP64
    g, ctx = pair(24, 16, 8, 4.0, lz=2 * np.pi * 8, policy="twothirds")
    r, phi, z = g.nodes3()
    s0 = O.to_flat(g, O.forward(g, W.fkpp_seed(r, phi, z)))
    ctx.implicit_setup(1.0, 1e-2)
    a = to_gpu_spec(s0)
    pa = ctx.new_spec()
    ctx.advance(B.NONLIN_FKPP, [1.0], a, pa, 10, True)
    b = to_gpu_spec(s0)
    pb = ctx.new_spec()
    ctx.advance(B.NONLIN_FKPP, [1.0], b, pb, 4, True)
    saved = (b.cpu().numpy().copy(), pb.cpu().numpy().copy())
    b2, pb2 = to_gpu_spec(saved[0]), to_gpu_spec(saved[1])
    ctx.advance(B.NONLIN_FKPP, [1.0], b2, pb2, 6, False)
    assert np.array_equal(a.cpu().numpy(), b2.cpu().numpy())


@pytest.mark.parametrize("prec,tol", [(B.FP64, 1e-12), (B.FP32, 1e-6), (B.BF16X3, 1e-6)])
def test_fkpp_full_size_sampled(prec, tol):
    # The benchmarked 3-D Fisher-KPP workload at full size (Nr = Nphi = 128,
    # Nz = 64, ell = 4, Lz = 2 pi 8, two-thirds chops, dt = 1e-2), in the launch
    # configuration the benchmark times (Richardson start, then graph-replayed
    # AB-CN pairs): 5 steps against the oracle.
    nr, nphi, nz, ell, lz = 128, 128, 64, 4.0, 2 * np.pi * 8
    g, ctx = pair(nr, nphi, nz, ell, lz=lz, policy="twothirds", precision=prec)
    r, phi, z = g.nodes3()
    u0 = W.fkpp_seed(r, phi, z)
    if prec != B.FP64:
        u0 = u0.astype(np.float32).astype(np.float64)
    import torch
    state = ctx.forward(torch.as_tensor(u0, dtype=ctx.phys_dtype).cuda(), ctx.new_spec())
    prevA = ctx.new_spec()
    ctx.implicit_setup(1.0, 1e-2)
    ctx.advance(B.NONLIN_FKPP, [1.0], state, prevA, 5, True)
    st = O.Stepper(g, 1.0, 1e-2, nonlinear=O.fkpp_nonlinear(g, 1.0))
    ref, refA = st.run_abcn(O.forward(g, u0), 5)
    assert O.spec_rel_err(g, spec_from_gpu(g, state), ref) <= tol
    assert O.spec_rel_err(g, spec_from_gpu(g, prevA), refA) <= tol


def test_fkpp_fp32_per_step_error_along_trajectory():
    # Accuracy per result: from FP64 states of the full-size workload at t = 0, 5
    # and 10, one FP32 time step against one FP64 time step (same state, same
    # A^{j-1}) stays within 1e-6.  (Whole trajectories drift apart as e^{gamma t}
    # because u = 0 is linearly unstable under gamma u (1 - u); that amplification
    # is a property of the equation and is reported by the benchmark.)
    import torch
    nr, nphi, nz, ell, lz = 128, 128, 64, 4.0, 2 * np.pi * 8
    g = O.Grid(nr, nphi, nz, ell, lz=lz, policy="twothirds")
    c64 = B.Context(nr, nphi, nz, ell, lz=lz, precision=B.FP64, chop_policy=B.CHOP_TWOTHIRDS)
    c32 = B.Context(nr, nphi, nz, ell, lz=lz, precision=B.FP32, chop_policy=B.CHOP_TWOTHIRDS)
    for c in (c64, c32):
        c.implicit_setup(1.0, 1e-2)
    x, w, r = c64.nodes()
    phi = 2 * np.pi * np.arange(nphi) / nphi
    zz = lz * np.arange(nz) / nz
    u0 = W.fkpp_seed(r[None, None, :], phi[None, :, None], zz[:, None, None])
    s = c64.forward(torch.as_tensor(u0, dtype=torch.float64).cuda(), c64.new_spec())
    a = c64.new_spec()
    c64.advance(B.NONLIN_FKPP, [1.0], s, a, 2, True)
    for seg in (0, 500, 500):
        if seg:
            c64.advance(B.NONLIN_FKPP, [1.0], s, a, seg, False)
        s64, a64 = s.clone(), a.clone()
        s32, a32 = s.clone(), a.clone()
        c64.advance(B.NONLIN_FKPP, [1.0], s64, a64, 1, False)
        c32.advance(B.NONLIN_FKPP, [1.0], s32, a32, 1, False)
        e_state = O.spec_rel_err(g, O.from_flat(g, s32.cpu().numpy()), O.from_flat(g, s64.cpu().numpy()))
        e_nonl = O.spec_rel_err(g, O.from_flat(g, a32.cpu().numpy()), O.from_flat(g, a64.cpu().numpy()))
        # A = gamma u (1 - u) loses relative accuracy as u saturates (A -> 0 while
        # u stays O(1)): a transform error du gives dA = gamma (1 - 2u) du, so the
        # bar on A is 1e-6 times kappa_A = max|1 - 2u| ||u|| / ||u (1 - u)||.
        u = c64.backward(s, c64.new_phys()).cpu().numpy()
        kappa = np.max(np.abs(1 - 2 * u)) * np.linalg.norm(u) / np.linalg.norm(u * (1 - u))
        assert e_state <= 1e-6, (seg, e_state)
        assert e_nonl <= 1e-6 * max(1.0, kappa), (seg, e_nonl, kappa)


@pytest.mark.parametrize("nu_h,p", [(0.0, 8), (5e-7, 8)])
@pytest.mark.parametrize("step", [B.STEP_ABCN, B.STEP_FEBE_FULL])
def test_solve_variants_agree(nu_h, p, step):
    # the staged (factor rows in shared memory, 8-32 chains per warp) and lean
    # (packed factor records, 16 or 32 chains per warp) variants solve the same
    # systems in one summation order: bitwise equal, and within 1e-12 (or 2 kappa u
    # for the ill-conditioned hyperviscous systems) of the oracle
    g, ctx = pair(40, 16, 8, 1.5, lz=3.0, policy="twothirds")
    ctx.implicit_setup(0.3, 2e-2, nu_h=nu_h, p=p)
    s, A, Ap = (to_gpu_spec(rand_spec(g, k)) for k in (1, 2, 3))
    outs = []
    variants = ((0, 8), (0, 16), (0, 32), (2, 16), (2, 32))
    ctx.set_tuning("solve_seg", 0)
    for direct, cpw in variants:
        ctx.set_tuning("solve_direct", direct)
        ctx.set_tuning("solve_lean_cpw" if direct == 2 else "solve_cpw", cpw)
        outs.append(ctx.implicit_solve(step, s, A, Ap, ctx.new_spec()).cpu().numpy())
    ctx.device_status()
    for v, o in enumerate(outs[1:], 1):
        assert np.array_equal(o, outs[0]), (variants[v], float(np.max(np.abs(o - outs[0]))))
    st = O.Stepper(g, 0.3, 2e-2, nu_h=nu_h, p=p)
    c = 1e-2 if step == B.STEP_ABCN else 2e-2
    kappa = max(np.linalg.cond(np.eye(L.shape[0]) - c * L) for L in st.L.values())
    tol = max(1e-12, 2.0 * kappa * 2.0 ** -53)
    S, Af, Apf = (O.from_flat(g, rand_spec(g, k)) for k in (1, 2, 3))
    ref = st.abcn(S, Af, Apf) if step == B.STEP_ABCN else st.febe(S, False, Af)
    assert O.spec_rel_err(g, O.from_flat(g, outs[0]), ref) <= tol


@pytest.mark.parametrize("grid", [(40, 16, 8, 1.5), (96, 32, 16, 1.0), (128, 128, 64, 4.0),
                                  (33, 16, 8, 1.0),    # shortest chain 28 rows: 8 segments fall back to 4
                                  (16, 8, 4, 1.0),     # only m = 0 (16 rows) cut in 4, m = 1, 2 staged
                                  (48, 128, 4, 1.0)])  # M = 43: m < 17 cut in 8 segments, the rest staged
@pytest.mark.parametrize("step", [B.STEP_FEBE_HALF, B.STEP_FEBE_FULL, B.STEP_ABCN])
def test_segmented_solve(grid, step):
    # half width 2: the chains cut into 4 or 8 row segments solved side by side, entry
    # states fixed by the precomputed influence data (orders whose chains are too
    # short for the segments go to the staged recurrence); same systems as the
    # staged recurrence, sums in another order: within 1e-12 of the oracle and of it
    nr, nphi, nz, ell = grid
    g, ctx = pair(nr, nphi, nz, ell, lz=3.0, policy="twothirds")
    dt, nu = 2e-2, 0.3
    ctx.implicit_setup(nu, dt)
    s, A, Ap = (rand_spec(g, k) for k in (7, 8, 9))
    outs = []
    for seg in (4, 8, 0):
        ctx.set_tuning("solve_seg", seg)
        outs.append(ctx.implicit_solve(step, to_gpu_spec(s), to_gpu_spec(A), to_gpu_spec(Ap),
                                       ctx.new_spec()).cpu().numpy())
    for o in outs[:2]:
        assert np.linalg.norm(o - outs[2]) <= 1e-13 * np.linalg.norm(outs[2])
    st = O.Stepper(g, nu, dt)
    S, AA, AP = (O.from_flat(g, v) for v in (s, A, Ap))
    ref = st.abcn(S, AA, AP) if step == B.STEP_ABCN else st.febe(S, step == B.STEP_FEBE_HALF, AA)
    assert O.spec_rel_err(g, O.from_flat(g, outs[0]), ref) <= 1e-12
    ctx.timing(True)
    ctx.implicit_solve(step, to_gpu_spec(s), to_gpu_spec(A), to_gpu_spec(Ap), ctx.new_spec())
    assert ctx.timing_read()["band_solve"][0] == 1
    ctx.timing(False)


@pytest.mark.parametrize("prec", [B.FP32, B.BF16X3])
@pytest.mark.parametrize("grid", [(128, 128, 64, 4.0), (48, 128, 4, 1.0), (16, 8, 4, 1.0)])
def test_segmented_solve_double_float(grid, prec, record):
    # FP32 / BF16x3 forms: the pivot-free segmented solve runs in double-float
    # arithmetic (hi + lo FP32 pairs, unit roundoff about 2^-47 per multiply-add against
    # 2^-53); against the FP64 recurrence of the same context and against the oracle,
    # the bound is the FP64 test's 2 kappa u with u = 2^-47, at least 1e-11
    nr, nphi, nz, ell = grid
    g, ctx = pair(nr, nphi, nz, ell, lz=3.0, policy="twothirds", precision=prec)
    dt, nu = 2e-2, 0.3
    ctx.implicit_setup(nu, dt)
    s, A, Ap = (rand_spec(g, k) for k in (17, 18, 19))
    st = O.Stepper(g, nu, dt)
    S, AA, AP = (O.from_flat(g, v) for v in (s, A, Ap))
    c = 0.5 * dt * nu
    kappa = max(np.linalg.cond(np.eye(L.shape[0]) - c * L) for L in st.L.values())
    tol = max(1e-11, 2.0 * kappa * 2.0 ** -47)
    for step in (B.STEP_ABCN, B.STEP_FEBE_HALF):
        outs = []
        for dfm in (1, 0):
            ctx.set_tuning("solve_df", dfm)
            outs.append(ctx.implicit_solve(step, to_gpu_spec(s), to_gpu_spec(A), to_gpu_spec(Ap),
                                           ctx.new_spec()).cpu().numpy())
        assert np.all(np.isfinite(outs[0]))
        assert np.linalg.norm(outs[0] - outs[1]) <= tol * np.linalg.norm(outs[1])
        ref = st.abcn(S, AA, AP) if step == B.STEP_ABCN else st.febe(S, True, AA)
        err = O.spec_rel_err(g, O.from_flat(g, outs[0]), ref)
        record("segmented_solve_df", grid=grid[:3], precision={B.FP32: "fp32", B.BF16X3: "bf16x3"}[prec],
               step=step, rel_err=err, fp64_form_err=O.spec_rel_err(g, O.from_flat(g, outs[1]), ref), tol=tol)
        assert err <= tol
    ctx.set_tuning("solve_df", 1)


def test_fkpp_plane_reuse_bitwise_and_split_count():
    # BF16x3 Fisher-KPP: within one mlx_advance call the segmented solve writes the
    # split planes of its output and the next step's backward contraction takes
    # them; the trajectory is bitwise that of splitting every step, and the split
    # kernel runs only for the Richardson start, the call's first pair and the odd
    # trailing step
    g, ctx = pair(40, 32, 16, 2.0, lz=2 * np.pi * 4, policy="twothirds", precision=B.BF16X3)
    r, phi, z = g.nodes3()
    s0 = O.to_flat(g, O.forward(g, W.fkpp_seed(r, phi, z)))
    ctx.implicit_setup(1.0, 1e-2)
    outs, splits = [], []
    for reuse in (1, 0):
        ctx.set_tuning("plane_reuse", reuse)
        state = to_gpu_spec(s0)
        prev = ctx.new_spec()
        ctx.timing(1)
        ctx.advance(B.NONLIN_FKPP, [1.0], state, prev, 21, True)
        kt = ctx.timing_read()
        ctx.timing(0)
        splits.append(kt.get("legendre_split", (0, 0.0))[0])
        state2 = to_gpu_spec(s0)
        prev2 = ctx.new_spec()
        ctx.advance(B.NONLIN_FKPP, [1.0], state2, prev2, 21, True)     # graph-replayed
        outs.append((state.cpu().numpy(), state2.cpu().numpy()))
    assert np.all(np.isfinite(outs[0][0]))
    assert np.array_equal(outs[0][0], outs[1][0])        # timing mode 1, reuse on / off
    assert np.array_equal(outs[0][1], outs[1][1])        # graphs, reuse on / off
    assert np.array_equal(outs[0][0], outs[0][1])        # direct launches = graphs
    # start (2 evaluations) + 20 AB-CN steps = 10 pairs: 2 + 1 with reuse, 2 + 20 without
    assert splits == [3, 22], splits
