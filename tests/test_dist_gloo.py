"""The multi-rank host logic on CPU: two gloo ranks reduce a timed run
(maximum elapsed time, summed work and launches) and compute the same
cost-balanced assignment of independent chains without communicating; the
assignment covers every chain once with loads within one chain's cost."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2601_16734_gb300.shard import chain_cost, reduce_run, shard_chains


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _specs():
    # the batched bench's shape family: N in 32..64, chi_max in {64, 128}
    return [(32 + (7 * k) % 33, [64, 128][(k * 5) % 2 if k % 3 else 1]) for k in range(64)]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = reduce_run(1.5 + rank, 10.0 * (rank + 1), 7 + rank)
        mine = shard_chains([chain_cost(n, chi) for n, chi in _specs()], world, rank)
        q.put((rank, res, mine))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_shard():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    for _, res, _ in got:
        assert res == (2.5, 30.0, 15)  # max(1.5, 2.5), 10 + 20, 7 + 8
    a, b = got[0][2], got[1][2]
    assert sorted(a + b) == list(range(64)) and not set(a) & set(b)
    # each rank's own computation agrees with what the other rank computed for it
    costs = [chain_cost(n, chi) for n, chi in _specs()]
    assert a == shard_chains(costs, 2, 0) and b == shard_chains(costs, 2, 1)


@pytest.mark.parametrize("world", [1, 2, 3, 5, 8])
def test_shard_covers_and_balances(world):
    costs = [chain_cost(n, chi) for n, chi in _specs()]
    parts = [shard_chains(costs, world, r) for r in range(world)]
    flat = sorted(k for p in parts for k in p)
    assert flat == list(range(len(costs)))
    loads = [sum(costs[k] for k in p) for p in parts]
    assert max(loads) - min(loads) <= max(costs)


def test_single_process_reduction_is_local():
    assert reduce_run(3.0, 4.0, 5) == (3.0, 4.0, 5)
    with pytest.raises(ValueError):
        shard_chains([1.0], 2, 2)
