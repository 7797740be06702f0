"""Multi-process host logic of bench.py's replica runs on CPU: two gloo ranks on
127.0.0.1 (no GPU).  The timed region's figure is the slowest rank's, the whole-job
value of N independent replicas is that time divided by N, counts add over ranks, and
every rank leaves the barrier."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, _ = bench.dist_env()
        t_local = 1.0 + 0.5 * rank            # per-step seconds measured by this rank
        t = bench.max_over_ranks(t_local, got_ws)
        n = bench.sum_over_ranks(10 * (rank + 1), got_ws)
        bench.rank_barrier(got_ws)
        out.put((got_rank, t, bench.replica_value(t, got_ws), n))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_add_counts():
    ws = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for _, t, value, n in res:
        assert t == 1.5                  # the slower rank's time, on every rank
        assert value == 0.75             # two replica steps complete in 1.5 s
        assert n == 30.0                 # 10 + 20


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.sum_over_ranks(7, 1) == 7.0
    assert bench.replica_value(2.5, 1) == 2.5
    bench.rank_barrier(1)
