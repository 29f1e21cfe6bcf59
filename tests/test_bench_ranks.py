"""The multi-rank reduction of bench.py on CPU (gloo, world size 2): every rank gets
the whole-job rate from the slowest rank's time, as a run over N GPUs reports it
(independent replicas, no data-path collective)."""

import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [200.0, 250.0][rank]          # the second rank is the slower one
    rate, slowest = bench.whole_job_rate(local_ms, 1000, world)
    with open(os.path.join(out_dir, "r%d" % rank), "w") as f:
        f.write("%r %r" % (rate, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_rate_max_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    ctx = mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=False,
                             start_method="spawn")
    while not ctx.join(timeout=120):
        pass
    for rank in range(2):
        rate, slowest = (float(v) for v in open(tmp_path / ("r%d" % rank)).read().split())
        assert slowest == 250.0
        assert rate == pytest.approx(2 * 1000 / 0.25)


def test_whole_job_rate_single_rank():
    import bench
    rate, slowest = bench.whole_job_rate(500.0, 100, 1)
    assert slowest == 500.0 and rate == pytest.approx(200.0)
