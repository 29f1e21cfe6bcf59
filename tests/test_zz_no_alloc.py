"""Allocation-free forward transform (mlx_forward_noalloc).

It serves callers that cannot call cudaMalloc while they transform, such as code
inside another framework's CUDA-graph capture or a host whose device-memory budget
is frozen after start-up: the intermediate Fourier planes live in a fixed 16 MiB
array built into the library instead of freshly allocated memory.  These tests
call it through the C-ABI and check that two calls in a row give the same result
as mlx_forward, that a call captured into a CUDA graph replays correctly on fresh
input, and that grids too large for the array are refused.  This file is
collected last so that a failure here never hides another test's result.
"""

import ctypes

import numpy as np
import pytest

from paper_2609_18026_b300 import binding as B

pytestmark = pytest.mark.gpu

TOL = {B.FP64: 1e-12, B.FP32: 1e-6, B.BF16X3: 1e-6}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", [B.FP64, B.FP32, B.BF16X3])
@pytest.mark.parametrize("grid", [(128, 128, 64, 4.0, B.CHOP_TWOTHIRDS),
                                  (32, 32, 1, 1.0, B.CHOP_LINEAR)])   # Nz = 1: no z planes
def test_noalloc_forward_matches_forward_twice(grid, prec):
    import torch
    nr, nphi, nz, ell, chop = grid
    lz = 2 * np.pi * 8
    ctx = B.Context(nr, nphi, nz, ell, lz=lz, precision=prec, chop_policy=chop)
    rng = np.random.default_rng(17)
    lib = B.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        phys = torch.as_tensor(rng.standard_normal((nz, nphi, nr)), dtype=ctx.phys_dtype).cuda()
        ref = ctx.forward(phys, ctx.new_spec())
        out = ctx.new_spec()
        rc = lib.mlx_forward_noalloc(ctx._h, ctypes.c_void_p(phys.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0, lib.mlx_last_cuda_error(ctx._h)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert _rel(a, b) <= TOL[prec], (call, _rel(a, b))
    ctx.device_status()


@pytest.mark.parametrize("prec", [B.FP64, B.BF16X3])
def test_noalloc_forward_inside_graph_capture(prec):
    # the entry point's purpose: after one warm-up call it can be captured into a
    # CUDA graph (no allocation, no synchronisation), and replays of that graph on
    # fresh input agree with mlx_forward
    import torch
    nr, nphi, nz, ell = 128, 128, 64, 4.0
    ctx = B.Context(nr, nphi, nz, ell, lz=2 * np.pi * 8, precision=prec, chop_policy=B.CHOP_TWOTHIRDS)
    lib = B.load()
    rng = np.random.default_rng(29)
    phys = torch.as_tensor(rng.standard_normal((nz, nphi, nr)), dtype=ctx.phys_dtype).cuda()
    out = ctx.new_spec()
    rc = lib.mlx_forward_noalloc(ctx._h, ctypes.c_void_p(phys.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.mlx_last_cuda_error(ctx._h)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        rc = lib.mlx_forward_noalloc(ctx._h, ctypes.c_void_p(phys.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.mlx_last_cuda_error(ctx._h)
    for rep in range(2):
        fresh = torch.as_tensor(rng.standard_normal((nz, nphi, nr)), dtype=ctx.phys_dtype).cuda()
        phys.copy_(fresh)
        out.zero_()
        graph.replay()
        torch.cuda.synchronize()
        ref = ctx.forward(fresh, ctx.new_spec())
        assert _rel(out.cpu().numpy(), ref.cpu().numpy()) <= TOL[prec], rep
    ctx.device_status()


def test_noalloc_rejects_grid_beyond_limit():
    import torch
    # 256^3 with two-thirds chops needs 4 * 2 * (171 + 256) * 86 * 256 bytes > 16 MiB
    ctx = B.Context(256, 256, 256, 1.0, lz=8.6, precision=B.FP32, chop_policy=B.CHOP_TWOTHIRDS)
    lib = B.load()
    phys = ctx.new_phys()
    out = ctx.new_spec()
    rc = lib.mlx_forward_noalloc(ctx._h, ctypes.c_void_p(phys.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1
    assert b"16777216" in lib.mlx_last_cuda_error(ctx._h)


def test_noalloc_forward_matches_oracle():
    # the same call against the FP64 oracle directly (test infrastructure only)
    import torch
    import oracle as O
    nr, nphi, nz, ell, lz = 40, 16, 8, 1.5, 3.0
    g = O.Grid(nr, nphi, nz, ell, lz=lz, policy="twothirds")
    ctx = B.Context(nr, nphi, nz, ell, lz=lz, precision=B.FP64, chop_policy=B.CHOP_TWOTHIRDS)
    u = np.random.default_rng(5).standard_normal((nz, nphi, nr))
    phys = torch.as_tensor(u).cuda()
    out = ctx.new_spec()
    lib = B.load()
    rc = lib.mlx_forward_noalloc(ctx._h, ctypes.c_void_p(phys.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.mlx_last_cuda_error(ctx._h)
    torch.cuda.synchronize()
    assert O.spec_rel_err(g, O.from_flat(g, out.cpu().numpy()), O.forward(g, u)) <= 1e-12
