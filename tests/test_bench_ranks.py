"""The multi-replica path of bench.py on CPU: two gloo ranks with different
timed regions must both report the slowest rank's time and the whole job's
throughput (instances of all ranks over that time)."""
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


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [800.0, 1000.0][rank]
    total, value = bench.job_throughput(ms, 5, world, dist, device="cpu")
    q.put((rank, total, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_report_max_time_and_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, value in got:
        assert total == 1000.0
        assert value == pytest.approx(2 * 5 / 1.0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.job_throughput(500.0, 3, 1) == (500.0, 6.0)
