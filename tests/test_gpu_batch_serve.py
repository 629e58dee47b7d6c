"""Batched and served forms: many independent hypergraphs partitioned concurrently on one GPU
must give exactly what the oracle (and the one-at-a-time path) gives for each of them."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    yield


def mixed_instances(n, seed=0):
    """Small instances of both workload shapes (netlist-like and row-net)."""
    out = []
    rng = np.random.default_rng(seed)
    for i in range(n):
        if i % 3 == 2:
            rows = int(rng.integers(800, 6000))
            out.append(synth.rownet(rows, rows, seed=4_000_000 + i))
        else:
            out.append(synth.c3_instance(i, N=int(rng.integers(1000, 12000))))
    return out


def test_batch_matches_oracle_and_solo():
    import paper_2012_13618_gb300 as bp
    graphs = mixed_instances(24)
    params = [dict(k=[2, 2, 4][i % 3], eps=0.05, policy="LDH", levels=25, iters=2)
              for i in range(len(graphs))]
    parts, st = bp.partition_batch(graphs, params, workers=6)
    for i, g in enumerate(graphs):
        hr = oracle.Hypergraph.from_dict(g)
        ref, rst = oracle.partition(hr, params[i]["k"], 0.05, "LDH", 25, 2)
        assert np.array_equal(parts[i], ref), i
        assert st[i] == rst
    # the same instance alone through the plain path
    with bp.create_from(graphs[5]) as h:
        solo, _ = h.partition(params[5]["k"], 0.05, "LDH", 25, 2)
    assert np.array_equal(solo, parts[5])


def test_batch_is_deterministic_under_different_worker_counts():
    import paper_2012_13618_gb300 as bp
    graphs = mixed_instances(12, seed=1)
    p = dict(k=2, eps=0.05, policy="HDH", levels=25, iters=2)
    a, _ = bp.partition_batch(graphs, p, workers=1)
    b, _ = bp.partition_batch(graphs, p, workers=8)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_server_mixed_requests_same_as_alone():
    import paper_2012_13618_gb300 as bp
    graphs = mixed_instances(18, seed=2)
    ks = [2, 4, 16]
    refs = []
    for i, g in enumerate(graphs):
        refs.append(oracle.partition(oracle.Hypergraph.from_dict(g), ks[i % 3], 0.05, "LDH", 25, 2))
    # a budget that admits only a few requests at a time forces queueing and overlap
    budget = 3 * max(64 * int(g["hoff"][-1]) + 96 * (g["E"] + g["N"]) + (8 << 20) for g in graphs)
    rng = np.random.default_rng(5)
    with bp.Server(hbm_budget_bytes=budget, workers=4) as srv:
        tickets = []
        for i, g in enumerate(graphs):
            tickets.append(srv.submit(g, k=ks[i % 3], eps=0.05, policy="LDH", levels=25, iters=2))
            time.sleep(float(rng.exponential(0.002)))
        for i, t in enumerate(tickets):
            parts, st, qms, rms = srv.wait(t)
            assert np.array_equal(parts, refs[i][0]), i
            assert st == refs[i][1]
            assert qms >= 0 and rms > 0


def test_server_rejects_request_above_budget():
    import paper_2012_13618_gb300 as bp
    g = synth.c3_instance(0, N=5000)
    with bp.Server(hbm_budget_bytes=1 << 20, workers=2) as srv:
        t = srv.submit(g, k=2, eps=0.05)
        parts, st, _, _ = srv.wait(t)
        assert st == bp.ERR_OOM
