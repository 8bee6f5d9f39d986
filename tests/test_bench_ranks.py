"""Host logic of bench.py's multi-rank path, on CPU with two gloo ranks: every
rank works on its own series (distinct seeds, no data-path collective), the
job time is the maximum over ranks, and the whole-job rate counts the units of
all ranks over that time."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 37.5 * rank  # the ranks finish at different times
        results[rank] = (bench.rank_seed(3, rank), bench.max_over_ranks(ms, world),
                         bench.job_rate(world, 10, bench.max_over_ranks(ms, world) / 1e3))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_their_own_series():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    world, port = 2, _free_port()
    with ctx.Manager() as m:
        results = m.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, results)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(results)
    seeds = [res[r][0] for r in range(world)]
    assert len(set(seeds)) == world
    for r in range(world):
        assert res[r][1] == pytest.approx(137.5)
        assert res[r][2] == pytest.approx(2 * 10 / 0.1375)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_rate(1, 2057, 7.2) == pytest.approx(2057 / 7.2)
    assert bench.rank_seed(3, 0) == 3
