"""The multi-rank path of bench.py on two gloo ranks (CPU): spectra are independent,
so the ranks exchange nothing but the barrier and the max-over-ranks step time,
and the reported value is the units of all ranks over the slowest rank's time."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        barrier, max_over_ranks = bench.make_collectives(ws, torch.device("cpu"))
        barrier()
        ms = max_over_ranks(40.0 + 5.0 * rank)          # the last rank is the slowest
        q.put((rank, ms, bench.aggregate_value(1000, ws, 4, ms)))
        barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_report_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=90) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert [r for r, _, _ in out] == [0, 1]
    for _, ms, value in out:
        assert ms == 45.0
        assert value == pytest.approx(2 * 1000 * 4 / 45e-3)


def test_single_rank_collectives_are_local():
    import torch

    import bench
    barrier, max_over_ranks = bench.make_collectives(1, torch.device("cpu"))
    barrier()
    assert max_over_ranks(3.5) == 3.5
    assert bench.aggregate_value(10, 1, 2, 4.0) == pytest.approx(10 * 2 / 4e-3)
