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


def test_single_rank_needs_no_process_group():
    assert replicas.max_over_ranks(3.0, 1) == 3.0
    assert replicas.whole_job_rate(10.0, 1, 2.0) == 5.0
