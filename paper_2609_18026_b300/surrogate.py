"""Training and evaluation of the learned vortex surrogate (no counterpart in the paper).

The surrogate advances the two-field vortex state s = (psi, chi) of the
counter-rotating pair (Sec. 5.3 workload at Nr = Nphi = Nz = 64) by nsub = 10
time steps per call:  s' = E^10 s + sigma_out f(s / sigma_in), with E the linear
AB-CN propagator and f the 4-layer width-64 network of the CUDA library
(mlx_sur_*).  Everything numerical runs in that library: the solver windows that
make the data, the propagator, the scale statistics, the sample assembly, the
forward and backward passes, Adam and the judged advance.  This module only
sequences those calls and moves device pointers.

Data.  A trajectory starts from one seeded pair (workloads.surrogate_trajectories)
and chains `windows` solver windows S^10 (Richardson start, then AB-CN; the same
map the judge applies), giving pairs (s^j, S^10(s^j)).

Usage:  python -m paper_2609_18026_b300.surrogate --trajectories 2000
"""

import argparse
import json
import math
import time

import numpy as np

from . import binding as B
from . import workloads as W

# The surrogate's workload: the vortex pair (circulation 2 pi, core radius about
# 0.2, separation about 1, axial period 8.6 b) at 64^3 in the frame moving with
# the pair (U0 e_y, U0 = -Gamma / (2 pi b) = -1).
CONFIG = dict(nr=64, nphi=64, nz=64, ell=1.0, lz=8.6, nu=1e-3, nu_h=0.0, p=8, dt=5e-4, U0=-1.0,
              nsub=10, windows=20, width=64, precision=B.BF16X3)


def make_context(cfg=CONFIG):
    ctx = B.Context(cfg["nr"], cfg["nphi"], cfg["nz"], cfg["ell"], lz=cfg["lz"], precision=cfg["precision"],
                    chop_policy=B.CHOP_TWOTHIRDS)
    ctx.vortex_setup()
    ctx.implicit_setup(cfg["nu"], cfg["dt"], nu_h=cfg["nu_h"], p=cfg["p"])
    return ctx


def initial_state(ctx, cfg, prm, torch):
    """(psi, chi) of one pair: psi = -lap_h^-1 omega_z, chi = 0."""
    x, w, r = ctx.nodes()
    phi = 2 * math.pi * np.arange(ctx.nphi) / ctx.nphi
    z = cfg["lz"] * np.arange(ctx.nz) / ctx.nz
    om = W.vortex_pair_omega(r[None, None, :], phi[None, :, None], z[:, None, None], lz=cfg["lz"],
                             b=prm["b"], a=prm["a"], amp=prm["amp"], incl_deg=prm["incl_deg"])
    ws = ctx.forward(torch.as_tensor(om, dtype=ctx.phys_dtype, device="cuda"), ctx.new_spec())
    s = torch.zeros(2 * ctx.n_spec, dtype=torch.complex128, device="cuda")
    ctx.lap_h_solve(-ws, s[:ctx.n_spec])
    return s


def trajectory(ctx, cfg, prm, torch, scratch=None):
    """States s^0 .. s^windows of one trajectory, [windows + 1][2 n_spec] complex128."""
    nw = cfg["windows"]
    out = torch.empty((nw + 1, 2 * ctx.n_spec), dtype=torch.complex128, device="cuda")
    s = initial_state(ctx, cfg, prm, torch)
    out[0] = s
    A = scratch if scratch is not None else torch.zeros_like(s)
    for j in range(nw):
        ctx.advance(B.NONLIN_VORTEX, [cfg["U0"]], s, A, cfg["nsub"], True)
        out[j + 1] = s
    return out


def build_dataset(ctx, sur, cfg, params, torch, n_fit=64, in_floor=1e-3, out_floor=0.0, log=None):
    """Fit the scales on the first n_fit trajectories, then fill X (BF16) and T
    (FP32), [len(params) * windows][D], pair by pair.  Per-coefficient output
    scales (out_floor < 1) keep the network's error spectrum in proportion to the
    remainder's own: coefficients that the solver leaves at zero (by the pair's
    mirror symmetry) get no correction, and small high-order ones (whose vorticity
    carries a factor of about n^2) are not swamped by errors sized for the large
    ones.  The loss weights (sigma_out_i^2) keep the objective the judge's norm."""
    nw, nsub = cfg["windows"], cfg["nsub"]
    scratch = torch.zeros(2 * ctx.n_spec, dtype=torch.complex128, device="cuda")
    t0 = time.perf_counter()
    for prm in params[:n_fit]:
        tr = trajectory(ctx, cfg, prm, torch, scratch)
        for j in range(nw):
            sur.observe(ctx, tr[j], tr[j + 1], nsub)
    sur.finalize_scales(in_floor, out_floor)
    n = len(params) * nw
    X = torch.empty((n, sur.D), dtype=torch.bfloat16, device="cuda")
    T = torch.empty((n, sur.D), dtype=torch.float32, device="cuda")
    for i, prm in enumerate(params):
        tr = trajectory(ctx, cfg, prm, torch, scratch)
        for j in range(nw):
            k = i * nw + j
            sur.make_pair(ctx, tr[j], tr[j + 1], nsub, X[k], T[k])
        if log and (i + 1) % 200 == 0:
            torch.cuda.synchronize()
            log("trajectories %d/%d (%.1f s)" % (i + 1, len(params), time.perf_counter() - t0))
    torch.cuda.synchronize()
    return X, T, time.perf_counter() - t0


def train(sur, X, T, n_train, torch, epochs=40, batch=128, lr=1e-3, lr_final=1e-5, seed=0, log=None):
    """Adam on the rows [0, n_train) of (X, T), cosine learning-rate decay.
    Returns the per-epoch mean losses and the wall time."""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    steps_per_epoch = max(1, n_train // batch)
    total = epochs * steps_per_epoch
    losses = torch.zeros(total, dtype=torch.float32, device="cuda")
    hist = []
    t0 = time.perf_counter()
    k = 0
    for ep in range(epochs):
        perm = torch.randperm(n_train, generator=g, device="cuda").to(torch.int32)
        for s in range(steps_per_epoch):
            idx = perm[s * batch:(s + 1) * batch]
            a = k / max(1, total - 1)
            lr_k = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * a))
            sur.train_step(X, T, idx, lr_k, losses[k:k + 1])
            k += 1
        hist.append(float(losses[k - steps_per_epoch:k].mean().item()))
        if log:
            log("epoch %d loss %.3e" % (ep, hist[-1]))
    torch.cuda.synchronize()
    return hist, time.perf_counter() - t0


def _rel(a, b, torch):
    return float(torch.linalg.vector_norm(a - b).item() / torch.linalg.vector_norm(b).item())


def evaluate(ctx, sur, cfg, trajs, torch, tol=1e-4):
    """Held-out comparison against the solver's own windows.

    Per trajectory (states s^0..s^n of the solver):
      * one-window residuals ||pred(s^j) - s^{j+1}|| / ||s^{j+1}|| of the network
        (through the judged advance) and of the propagator alone (f = 0);
      * free-running chains of n calls without the judge, network and f = 0,
        and their error against s^n;
      * the judged chain (fallback on): accepted fraction and error against s^n."""
    nsub, U0 = cfg["nsub"], cfg["U0"]
    res_nn, res_0, acc = [], [], []
    chain_nn, chain_0, chain_j, acc_chain = [], [], [], []
    tmp = torch.empty_like(trajs[0][0])
    for tr in trajs:
        n = tr.shape[0] - 1
        for j in range(n):
            s = tr[j].clone()
            a, r = sur.advance(ctx, s, nsub, U0, True, tol)
            res_nn.append(r)
            acc.append(a)
            sur.propagate(ctx, tr[j], tmp, nsub)
            res_0.append(_rel(tmp, tr[j + 1], torch))
        s = tr[0].clone()
        for j in range(n):
            sur.advance(ctx, s, nsub, U0, False, tol)
        chain_nn.append(_rel(s, tr[n], torch))
        s = tr[0].clone()
        for j in range(n):
            sur.propagate(ctx, s, tmp, nsub)
            s.copy_(tmp)
        chain_0.append(_rel(s, tr[n], torch))
        s = tr[0].clone()
        na = 0
        for j in range(n):
            a, _ = sur.advance(ctx, s, nsub, U0, True, tol)
            na += int(a)
        chain_j.append(_rel(s, tr[n], torch))
        acc_chain.append(na / n)
    return dict(
        tol=tol,
        window_residual_nn_median=float(np.median(res_nn)), window_residual_nn_max=float(np.max(res_nn)),
        window_residual_prop_median=float(np.median(res_0)), window_residual_prop_max=float(np.max(res_0)),
        accepted_fraction=float(np.mean(acc)),
        chain_error_nn=float(np.median(chain_nn)), chain_error_prop=float(np.median(chain_0)),
        chain_error_judged=float(np.median(chain_j)), chain_accepted_fraction=float(np.mean(acc_chain)),
    )


def throughput(ctx, sur, cfg, s0, torch, calls=20, judge_every=0, tol=1e-4):
    """Time steps per second of (a) the plain solver in windows of nsub steps and
    (b) the surrogate, judged every `judge_every`-th call (0: never), from s0.
    CUDA events on the current stream around the whole sequence."""
    nsub, U0 = cfg["nsub"], cfg["U0"]
    st = torch.cuda.current_stream()
    A = torch.zeros_like(s0)

    def timed(fn):
        s = s0.clone()
        fn(s)                                   # warm-up (graph capture)
        s = s0.clone()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        nacc = fn(s)
        e1.record(st)
        torch.cuda.synchronize()
        return calls * nsub / (e0.elapsed_time(e1) / 1000.0), nacc

    def solver(s):
        for _ in range(calls):
            ctx.advance(B.NONLIN_VORTEX, [U0], s, A, nsub, True)
        return calls

    def surrogate(s):
        na = 0
        for c in range(calls):
            judge = judge_every > 0 and c % judge_every == 0
            a, _ = sur.advance(ctx, s, nsub, U0, judge, tol)
            na += int(a)
        return na

    sps_solver, _ = timed(solver)
    sps_sur, nacc = timed(surrogate)
    return dict(solver_steps_per_s=sps_solver, surrogate_steps_per_s=sps_sur, judge_every=judge_every,
                accepted_calls=nacc, calls=calls)


def run(n_traj=2000, n_test=None, epochs=40, batch=128, lr=1e-3, seed=20261203, cfg=CONFIG, log=print):
    """Full pipeline: data, training, held-out evaluation, throughput."""
    import torch
    torch.cuda.init()
    n_test = n_test if n_test is not None else max(1, n_traj // 10)
    params = W.surrogate_trajectories(n_traj, seed)
    ctx = make_context(cfg)
    D = 4 * ctx.n_spec
    sur = B.Surrogate(D, width=cfg["width"], bmax=max(batch, 1), seed=seed)
    n_tr = n_traj - n_test
    X, T, t_data = build_dataset(ctx, sur, cfg, params[:n_tr], torch, n_fit=min(64, n_tr), log=log)
    hist, t_train = train(sur, X, T, X.shape[0], torch, epochs=epochs, batch=batch, lr=lr, log=log)
    del X, T
    torch.cuda.empty_cache()
    scratch = torch.zeros(2 * ctx.n_spec, dtype=torch.complex128, device="cuda")
    trajs = [trajectory(ctx, cfg, p, torch, scratch) for p in params[n_tr:n_tr + min(n_test, 20)]]
    ev = evaluate(ctx, sur, cfg, trajs, torch)
    tp = [throughput(ctx, sur, cfg, trajs[0][0], torch, judge_every=j) for j in (0, 1, 10)]
    out = dict(trajectories=n_traj, test_trajectories=len(trajs), D=D, params=sur.nparam,
               data_s=t_data, train_s=t_train, final_loss=hist[-1], loss_history=hist[::max(1, len(hist) // 10)],
               eval=ev, throughput=tp)
    sur.close()
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--trajectories", type=int, default=2000)
    ap.add_argument("--test", type=int, default=None)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=128)
    ap.add_argument("--lr", type=float, default=1e-3)
    a = ap.parse_args()
    out = run(a.trajectories, a.test, a.epochs, a.batch, a.lr)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
