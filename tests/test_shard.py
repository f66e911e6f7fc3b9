"""Instance sharding of batches (paper_1903_06477_gb300/shard.py) on CPU: the
partition covers every instance once and is balanced, and two gloo ranks
gather each other's per-instance results in global order."""
import os
import socket

import pytest

from paper_1903_06477_gb300 import shard
from paper_1903_06477_gb300 import workloads as W

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _costs(count=300):
    return [shard.instance_cost(p) for p in W.c4_portfolios(count)]


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_partition_covers_and_balances(world):
    costs = _costs()
    parts = shard.partition(costs, world)
    assert len(parts) == world
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(costs)))
    ld = shard.loads(costs, parts)
    # longest-processing-time: no rank exceeds another by more than one instance's cost
    assert max(ld) - min(ld) <= max(costs)
    assert shard.partition(costs, world) == parts  # deterministic


def test_partition_edge_cases():
    assert shard.partition([], 2) == [[], []]
    assert shard.partition([5], 3) == [[0], [], []]
    assert shard.partition([1, 1, 1, 1], 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        shard.partition([1], 0)


def test_gather_single_process_and_errors():
    assert shard.gather([2, 0, 1], ["c", "a", "b"], 3) == ["a", "b", "c"]
    with pytest.raises(ValueError):
        shard.gather([0, 0], ["a", "b"], 2)
    with pytest.raises(ValueError):
        shard.gather([0], ["a"], 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    costs = [shard.instance_cost(p) for p in W.c4_portfolios(120)]
    parts = shard.partition(costs, world)
    mine = parts[rank]
    results = [(i, rank, costs[i]) for i in mine]  # stands in for (status, iters, pobj)
    got = shard.gather(mine, results, len(costs), dist)
    q.put((rank, parts, got))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_in_global_order():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, parts0, res0), (_, parts1, res1) = got
    assert parts0 == parts1
    assert res0 == res1
    owner = {i: r for r, p in enumerate(parts0) for i in p}
    assert [r[0] for r in res0] == list(range(120))
    assert all(r[1] == owner[r[0]] for r in res0)
