"""Multi-rank logic of the weak-scaling bench on the CPU: two gloo ranks.

Signals are independent, so ranks solve disjoint shards of one seeded batch and exchange
nothing on the data path; the job's time is the max over ranks and its solves the sum.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synthetic as S
    B = 3
    first = bench.shard_first(rank, B)
    w = S.c3(n_signals=B, first=first, N=32, K=64)
    # each rank's local numbers differ; the job takes the max time and the total solves
    t, n = bench.job_totals(1.0 + rank, 10 * (rank + 1), torch.device("cpu"))
    out.put((rank, first, w.Y, w.lam_ratio, t, n))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r, first, Y, lam, t, n = q.get(timeout=180)
        res[r] = (first, Y, lam, t, n)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import synthetic as S
    whole = S.c3(n_signals=6, N=32, K=64)
    for r in range(2):
        first, Y, lam, t, n = res[r]
        assert first == 3 * r
        # the shard is exactly the slice of the single-process batch: no overlap, no gap
        np.testing.assert_array_equal(Y, whole.Y[first:first + 3])
        np.testing.assert_array_equal(lam, whole.lam_ratio[first:first + 3])
        assert t == 2.0 and n == 30


def test_single_process_totals_are_local():
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import bench
    assert bench.job_totals(0.5, 7, torch.device("cpu")) == (0.5, 7)
    assert bench.shard_first(0, 4096) == 0 and bench.shard_first(3, 4096) == 12288


@pytest.mark.parametrize("world", [2])
def test_reference_arm_runs_on_rank_zero_only(world, monkeypatch, capsys):
    """Under torchrun only rank 0 runs the (CPU) reference arm; the others exit 0 silently."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", str(world))

    class A:
        steps, warmup, gpus = 1, 0, world
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
