"""The benchmark's multi-process path on the CPU (gloo, world size 2): every
rank reconstructs its own frame (different seeds, no data-path collective),
the timed region is the maximum over ranks, and the whole-job rate counts
every rank's units over that maximum."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    import bench
    from paper_1812_03358_b300 import inputs as I
    t = bench.max_over_ranks(1.0 + 0.5 * rank, "cpu")
    rate = bench.job_rate(100, 10, world, t)
    vol = I.Volume(8, 8, 8, 1.0, 1.0, 1.0)
    x = I.plume_field(vol, seed=bench.frame_seed(rank))
    q.put((rank, t, rate, float(x.sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    import torch.multiprocessing as mp
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    assert res[0][1] == res[1][1] == 1.5                  # max over ranks, seen by both
    assert res[0][2] == res[1][2] == 2 * 100 * 10 / 1.5   # whole-job rate
    assert res[0][3] != res[1][3]                         # independent frames


def test_single_rank_helpers_without_a_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, "cpu") == 3.25
    assert bench.job_rate(7, 3, 1, 2.0) == 10.5
    assert bench.frame_seed(0) != bench.frame_seed(1)
