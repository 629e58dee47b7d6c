"""Instance sharding across ranks (CPU, gloo, world size 2): every rank derives the same
longest-processing-time assignment, the shares cover every instance exactly once, and the
reported time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2012_13618_gb300 import shard


def test_assign_covers_and_balances():
    rng = np.random.default_rng(0)
    costs = rng.integers(1, 1000, size=257).tolist()
    for world in (1, 2, 3, 8):
        parts = shard.assign(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT bound: max load <= 4/3 of the optimum lower bound (+ one item)
        assert max(loads) <= sum(costs) / world + max(costs)
    assert shard.assign([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, costs, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard.my_share(costs, rank, world)
    t = 1.0 + rank  # this rank's time
    tmax = shard.max_over_ranks(t)
    q.put((rank, mine, tmax))
    dist.destroy_process_group()


def test_two_ranks_share_and_max_time():
    costs = [7, 3, 9, 1, 4, 4, 8, 2]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    shares = [r[1] for r in res]
    assert sorted(shares[0] + shares[1]) == list(range(len(costs)))
    assert shares == shard.assign(costs, 2)
    assert all(r[2] == 2.0 for r in res)


def _serve_worker(rank, world, port, costs, arrivals, q):
    # each rank serves its share of the request trace in arrival order (a single-server queue
    # simulated on the host: a request starts at max(arrival, previous completion)); nothing is
    # exchanged while serving, only the final span is reduced
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine, arr = shard.serve_share(costs, arrivals, rank, world)
    done = 0.0
    for i, a in zip(mine, arr):
        done = max(done, a) + costs[i] * 1e-3
    span = shard.max_over_ranks(done)
    slowest = shard.min_over_ranks(-done)
    q.put((rank, mine, arr, done, span, slowest))
    dist.destroy_process_group()


def test_two_ranks_serve_shares_of_one_trace():
    rng = np.random.default_rng(3)
    costs = rng.integers(1, 500, size=40).tolist()
    arrivals = np.cumsum(rng.exponential(0.05, size=40)).tolist()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_serve_worker, args=(r, 2, port, costs, arrivals, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    shares = [r[1] for r in res]
    assert sorted(shares[0] + shares[1]) == list(range(len(costs)))
    assert [sorted(s) for s in shares] == shard.assign(costs, 2)
    for _, mine, arr, _, _, _ in res:
        assert arr == [arrivals[i] for i in mine] and arr == sorted(arr)
    spans = [r[3] for r in res]
    assert all(r[4] == max(spans) for r in res)
    assert all(r[5] == -max(spans) for r in res)
