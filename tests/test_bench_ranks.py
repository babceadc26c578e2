"""The benchmark's multi-rank path on CPU: two gloo ranks, as torchrun starts
them, each with its own replica of the workload.  The job's step is the
slowest rank's (a max over the ranks) and its throughput counts every
rank's atoms; rank 0 alone reports it.  No GPU and no collective on the data
path: the replicas share nothing but this reduction of their timings."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_setup(None)
    ms = 1.5 + rank  # rank 1 is the slower one
    t = bench.max_over_ranks(dist, ms, "cpu")
    value = bench.job_throughput(w, 2000, t)
    dist.barrier()
    dist.destroy_process_group()
    out.put((r, local, w, t, value))


def test_two_gloo_ranks_report_the_slowest_step_and_all_atoms():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for k, (r, local, w, t, value) in enumerate(res):
        assert (r, local, w) == (k, k, 2)
        assert t == 2.5                      # the slower rank's step, on both ranks
        assert value == pytest.approx(2 * 2000 / 2.5e-3)


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 1.25, "cpu") == 1.25
    assert bench.job_throughput(1, 2000, 0.137) == pytest.approx(2000 / 0.137e-3)
