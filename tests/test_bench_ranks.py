"""The multi-rank path of bench.py on the CPU (gloo, world size 2): the job's time per step is
the slowest rank's, every rank sees it, and the whole-job throughput counts every rank's
replica (weak scaling).  The reference arm runs on rank 0 only."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench.dist_init()
    ms = bench.max_over_ranks(1.0 + 2.0 * rank, w)            # rank 1 is the slow one
    q.put((r, ms, bench.whole_job_mlups(w, 1000, ms)))
    dist.destroy_process_group()


def test_timing_is_the_max_over_ranks_and_value_counts_all_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    for _, ms, v in got:
        assert ms == 3.0
        assert v == pytest.approx(2 * 1000 / 3e-3 / 1e6)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.whole_job_mlups(1, 65536, 1.0) == pytest.approx(65.536)


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(gpus=2, steps=1, warmup=0)
    assert bench.run_reference(args, world=2, rank=1) == 0    # returns at once, no oracle work
