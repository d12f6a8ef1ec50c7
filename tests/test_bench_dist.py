"""The multi-rank path of bench.py on CPU: two gloo ranks (world size 2, one
process each, rendezvous on 127.0.0.1) reduce their step times to the
maximum, and the whole-job rate counts the work of every rank (replicas,
weak scaling)."""
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


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, w, "cpu")  # rank 1 is the slow one
        rate = bench.whole_job_rate(1.0e9, 3, ms, w)
        q.put((r, w, local, ms, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_maximum_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    for _, _, _, ms, rate in out:
        assert ms == pytest.approx(15.0)
        assert rate == pytest.approx(2 * 1.0e9 * 3 / 0.015)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5
    assert bench.whole_job_rate(2.0, 4, 1000.0, 1) == pytest.approx(8.0)
