"""The N > 1 bench path on CPU: two gloo ranks, each timing its own replica,
agree on the slowest rank's time, and the whole-job throughput counts every
rank's cells over that time (replicas, no exchange step)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 180.0][rank]
        dist.barrier()
        ms = bench.max_over_ranks(local_ms, dist, torch.device("cpu"))
        out.put((rank, ms, bench.job_throughput(1e9, world, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [180.0, 180.0]
    assert all(abs(r[2] - 2e9 / 0.18) < 1e-3 for r in res)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(42.0, None, None) == 42.0
    assert bench.job_throughput(5e8, 1, 500.0) == pytest.approx(1e9)
