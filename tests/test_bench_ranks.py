"""Multi-process aggregation of bench.py on CPU: two gloo ranks (replicas with
different work) report edges summed over ranks and times as the maximum over
ranks, as the whole-job value requires."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r: (r + 1) * 1000 edges in (r + 1) * 2.5 ms; e2e 10 (r + 1) edges in 0.1 (r + 1) s
    res = bench.aggregate_over_ranks((rank + 1) * 1000, (rank + 1) * 2.5, 10 * (rank + 1), 0.1 * (rank + 1), dist)
    out[rank] = res
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_edges_and_take_max_time():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        edges, ms, e2e_edges, e2e_s = out[r]
        assert edges == 3000.0 and ms == 5.0
        assert e2e_edges == 30.0 and abs(e2e_s - 0.2) < 1e-12


def test_single_process_is_identity():
    pytest.importorskip("torch")
    import bench
    assert bench.aggregate_over_ranks(7, 1.5, 3, 0.25) == (7.0, 1.5, 3.0, 0.25)
