"""The N-rank host logic of bench.py on CPU (two gloo ranks): the path shards as independent
replicas, so the only cross-rank steps are the barrier around the timed region and the
max-over-ranks time; the whole-job rate counts every rank's units over that time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR='127.0.0.1', MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group('gloo', rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        dist.barrier()
        ms = bench.max_over_ranks(100.0 + 50.0 * rank, dist, 'cpu')
        rate = bench.job_rate(1e6, ws, ms)
        out.put((r, ws, local, ms, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_rate():
    ctx = mp.get_context('spawn')
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 and r[2] == r[0] for r in res)
    assert all(r[3] == pytest.approx(150.0) for r in res)          # max over ranks
    assert all(r[4] == pytest.approx(2 * 1e6 / 0.150) for r in res)  # units of both ranks / slowest time


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(42.0, None, 'cpu') == 42.0
    assert bench.job_rate(10.0, 1, 1000.0) == pytest.approx(10.0)
