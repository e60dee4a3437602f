"""Host-side logic of bench.py without a GPU: aggregation over ranks (gloo,
world size 2, as torch.distributed.run would launch them), clock summaries."""

import datetime
import os
import socket

import pytest

import bench


def test_aggregate_value():
    assert bench.aggregate_value(100, 1, 0.5) == 200.0
    assert bench.aggregate_value(100, 4, 0.5) == 800.0


def test_summarize_clocks_window_and_reasons():
    t = datetime.datetime(2026, 1, 1, 12, 0, 0)
    fmt = lambda dt: dt.strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    lines = [
        f"{fmt(t)}, 1200, 2070, 300.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        f"{fmt(t + datetime.timedelta(seconds=1))}, 1900, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active",
        f"{fmt(t + datetime.timedelta(seconds=2))}, 1950, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    s = bench.summarize_clocks("\n".join(lines), (t + datetime.timedelta(seconds=0.5), t + datetime.timedelta(seconds=2.5)))
    assert s["samples_in_window"] == 2 and s["sm_mhz"] == 1925.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert bench.summarize_clocks("") is None


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    dist = bench.dist_init(world, "gloo")
    r, lr, w = bench.dist_env()
    slowest = bench.max_over_ranks(dist, 1.0 + r)      # rank 1 is the slow one
    bench.barrier(dist)
    q.put((r, w, slowest, bench.aggregate_value(100, w, slowest)))
    dist.destroy_process_group()


def test_two_rank_max_and_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 2, 2.0, 100.0), (1, 2, 2.0, 100.0)]
