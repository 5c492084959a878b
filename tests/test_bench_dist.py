"""The N > 1 path of bench.py on CPU: two gloo ranks.  The bench runs one independent
replica per rank (no data-path collective); what crosses ranks is the barrier around the
timed region and the max over ranks of the elapsed time.  The reference arm runs on rank 0
only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", world_size=world, rank=rank)
    bench.barrier(dist)
    elapsed = 1.0 + 0.5 * rank                     # this rank's own timed region
    out[rank] = bench.max_over_ranks(dist, elapsed)
    bench.barrier(dist)
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_max_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 1.5


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(ref_iters=35, warmup=3, steps=3)
    bench.run_reference(args, world=2, rank=1)     # a non-zero rank does no work
    assert capsys.readouterr().out == ""
