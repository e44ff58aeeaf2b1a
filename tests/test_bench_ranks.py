"""The benchmark's multi-rank path on CPU: two gloo ranks (one process each), the max-over-ranks
step time and the whole-job rate that bench.py reports, and distinct instances per rank."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    from paper_2201_05024_gb300 import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank times its own steps; rank 1 is the slow one
    own = [2.0 + rank, 1.0 + 0.5 * rank, 0.25]
    ms = bench.reduce_max(dist, own, "cpu")
    rate = bench.job_rate(world, 65536, ms[0])
    inst = synth.make_instance(4, 2, 8, 4, 10.0, instance=rank)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ms, rate, inst.rx_pilot.copy()))


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_slowest_rank_and_count_every_ranks_units():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=100) for _ in range(world))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, ms, rate, _ in res:
        assert ms == [3.0, 1.5, 0.25]                      # max over ranks, element by element
        assert rate == pytest.approx(2 * 65536 / 3.0e-3)   # both ranks' vectors in the slowest time
    assert not np.array_equal(res[0][3], res[1][3])        # independent instance per rank


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(None, [1.0, 2.0], "cpu") == [1.0, 2.0]
    assert bench.job_rate(1, 1000, 2.0) == pytest.approx(5e5)
