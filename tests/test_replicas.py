"""Two gloo ranks on CPU run the bookkeeping of a replicas run: the barrier,
the maximum of the per-rank times and the whole-job rate."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1908_08386_gb300 import replicas  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, size, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(size), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    r, n, local = replicas.init("gloo")
    assert (r, n, local) == (rank, size, rank)
    replicas.barrier(n)
    t = 1.5 + rank  # per-rank seconds
    slowest = replicas.max_over_ranks(t, n, device="cpu")
    rate = replicas.whole_job_rate(1000.0, n, slowest)
    out.put((rank, slowest, rate))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_rate():
    size, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, size, port, q)) for r in range(size)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(size))
    for rank, slowest, rate in res:
        assert slowest == 2.5
        assert rate == pytest.approx(1000.0 * 2 / 2.5)


def _shard_rank(rank, size, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(size), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    r, n, _ = replicas.init("gloo")
    costs = [5.0, 1.0, 4.0, 4.0, 2.0, 3.0, 1.0]
    mine = replicas.shard(costs, n)[r]
    # each rank "solves" its cavities: a row per cavity it holds
    rows = [(i, r, costs[i] * 10) for i in mine]
    everything = replicas.gather_rows(rows, n)
    out.put((rank, mine, everything))
    dist.destroy_process_group()


def test_sharded_cavities_are_gathered_on_every_rank():
    size, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_rank, args=(r, size, port, q)) for r in range(size)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(size))
    shards = [m for _, m, _ in res]
    assert sorted(shards[0] + shards[1]) == list(range(7))  # every cavity once
    assert res[0][2] == res[1][2]  # both ranks hold the same table
    table = sorted(res[0][2])
    assert [t[0] for t in table] == list(range(7)) and all(t[1] in (0, 1) for t in table)


def test_shard_balances_costs():
    costs = [9.0, 1.0, 4.0, 4.0, 2.0, 3.0, 1.0, 8.0]
    parts = replicas.shard(costs, 3)
    loads = [sum(costs[i] for i in p) for p in parts]
    assert sorted(i for p in parts for i in p) == list(range(8))
    assert max(loads) - min(loads) <= max(costs)
    assert replicas.shard(costs, 1) == [list(range(8))]


def test_single_rank_needs_no_process_group():
    assert replicas.max_over_ranks(3.0, 1) == 3.0
    assert replicas.whole_job_rate(10.0, 1, 2.0) == 5.0
    assert replicas.gather_rows([1, 2], 1) == [1, 2]
