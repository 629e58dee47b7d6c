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


def test_batch_deterministic_ten_runs():
    # the batched call (persistent block kernel for the k = 2 instances, worker pool for k = 4)
    # gives the same parts on ten calls, equal to the oracle's
    import paper_2012_13618_gb300 as bp
    graphs = mixed_instances(10, seed=7)
    params = [dict(k=[2, 2, 4][i % 3], eps=0.05, policy="LDH", levels=25, iters=2)
              for i in range(len(graphs))]
    first, st0 = bp.partition_batch(graphs, params, workers=4)
    for i, g in enumerate(graphs):
        ref, rst = oracle.partition(oracle.Hypergraph.from_dict(g), params[i]["k"], 0.05, "LDH", 25, 2)
        assert np.array_equal(first[i], ref) and st0[i] == rst, i
    for run in range(9):
        parts, st = bp.partition_batch(graphs, params, workers=[1, 4, 8][run % 3])
        assert np.array_equal(st, st0), run
        for a, b in zip(parts, first):
            assert np.array_equal(a, b), run


def test_server_mix_deterministic_ten_runs():
    # ten rounds of the same mixed request trace through one server: every result identical
    import paper_2012_13618_gb300 as bp
    graphs = mixed_instances(9, seed=8)
    ks = [2, 4, 16]
    refs = [oracle.partition(oracle.Hypergraph.from_dict(g), ks[i % 3], 0.05, "LDH", 25, 2)
            for i, g in enumerate(graphs)]
    with bp.Server(hbm_budget_bytes=8 << 30, workers=4) as srv:
        for run in range(10):
            tickets = [srv.submit(g, k=ks[i % 3], eps=0.05) for i, g in enumerate(graphs)]
            for i, t in enumerate(tickets):
                parts, st, _, _ = srv.wait(t)
                assert np.array_equal(parts, refs[i][0]) and st == refs[i][1], (run, i)


def test_server_rejects_request_above_budget():
    import paper_2012_13618_gb300 as bp
    g = synth.c3_instance(0, N=5000)
    with bp.Server(hbm_budget_bytes=1 << 20, workers=2) as srv:
        t = srv.submit(g, k=2, eps=0.05)
        parts, st, _, _ = srv.wait(t)
        assert st == bp.ERR_OOM


def _block_cases():
    rng = np.random.default_rng(9)
    out = []
    for i in range(40):
        kind = i % 5
        if kind == 0:
            out.append(synth.uniform(int(rng.integers(50, 3000)), int(rng.integers(50, 3000)), 2, 7, seed=100 + i))
        elif kind == 1:
            out.append(synth.c3_instance(500 + i, N=int(rng.integers(1000, 30000))))
        elif kind == 2:
            r = int(rng.integers(500, 8000))
            out.append(synth.rownet(r, r, seed=200 + i))
        elif kind == 3:  # weighted hyperedges, duplicate and single pins
            N, E = int(rng.integers(100, 2000)), int(rng.integers(100, 3000))
            deg = rng.integers(0, 9, size=E)
            hoff = np.zeros(E + 1, np.int32)
            hoff[1:] = np.cumsum(deg)
            out.append(dict(N=N, E=E, hoff=hoff, pins=rng.integers(0, N, size=int(hoff[-1])).astype(np.int32),
                            nw=rng.integers(1, 6, size=N).astype(np.int32),
                            hw=rng.integers(1, 2000, size=E).astype(np.int32)))
        else:  # degenerate: no hyperedges, or a handful of nodes
            N = int(rng.integers(1, 40))
            out.append(dict(N=N, E=0, hoff=np.zeros(1, np.int32), pins=np.zeros(0, np.int32), nw=None, hw=None))
    return out


def test_block_path_many_instances_match_oracle():
    import paper_2012_13618_gb300 as bp
    graphs = _block_cases()
    pols = ["LDH", "HDH", "LWD", "HWD", "RAND"]
    params = [dict(k=2, eps=[0.0, 0.05, 0.1, 0.3][i % 4], policy=pols[i % 5], levels=[25, 3, 0, 25][i % 4],
                   iters=[2, 1, 2, 0][i % 4]) for i in range(len(graphs))]
    parts, st = bp.partition_batch(graphs, params, workers=4)
    for i, g in enumerate(graphs):
        p = params[i]
        r = oracle.bisect(oracle.Hypergraph.from_dict(g), p["eps"], p["policy"], p["levels"], p["iters"],
                          keep_levels=False)
        assert np.array_equal(parts[i], r["side"].astype(np.int32)), i
        assert st[i] == r["status"], i


def test_block_path_deferral_falls_back(monkeypatch):
    # an arena too small for the larger instances defers them to the single-instance path
    import paper_2012_13618_gb300 as bp
    graphs = [synth.c3_instance(700 + i, N=n) for i, n in enumerate([2000, 40000, 3000, 60000])]
    p = dict(k=2, eps=0.05, policy="LDH", levels=25, iters=2)
    want = [oracle.bisect(oracle.Hypergraph.from_dict(g), 0.05, "LDH", 25, 2, keep_levels=False)["side"]
            for g in graphs]
    monkeypatch.setenv("BIPART_BLOCK_ARENA_MB", "8")
    parts, st = bp.partition_batch(graphs, p, workers=2)
    for a, b in zip(parts, want):
        assert np.array_equal(a, b.astype(np.int32))


def test_design_space_sweep_matches_oracle_and_frontier():
    from paper_2012_13618_gb300 import sweep
    g = synth.uniform(2500, 2600, 2, 6, seed=31)
    res, front = sweep.sweep(g, levels=(3, 25), iters=(0, 2), policies=("LDH", "RAND"), eps=0.1,
                             repeats=1)
    hr = oracle.Hypergraph.from_dict(g)
    for r in res:
        ref = oracle.bisect(hr, 0.1, r["policy"], r["levels"], r["iters"], keep_levels=False)
        assert np.array_equal(r["parts"], ref["side"].astype(np.int32))
        assert r["cut"] == oracle.cut_bisection(hr, ref["side"])
    pts = [(r["ms"], r["cut"]) for r in res]
    assert front and all(not any(pts[j][0] <= pts[i][0] and pts[j][1] <= pts[i][1] and pts[j] != pts[i]
                                 for j in range(len(pts))) for i in front)


def test_batch_general_k_matches_single():
    # the worker pool runs k = 3 / 6 (adaptive) requests exactly as bipart_partition does
    import paper_2012_13618_gb300 as bp
    graphs = [synth.uniform(2000 + 300 * i, 2100 + 300 * i, 2, 6, seed=60 + i) for i in range(4)]
    params = [dict(k=3, eps=0.05, policy="LDH", levels=25, iters=2, adaptive_eps=bool(i % 2))
              for i in range(2)] + [dict(k=6, eps=0.05, policy="LDH", levels=25, iters=2,
                                         adaptive_eps=bool(i % 2)) for i in range(2)]
    parts, sts = bp.partition_batch(graphs, params, workers=3)
    for i, g in enumerate(graphs):
        ref, rst = oracle.partition(oracle.Hypergraph.from_dict(g), params[i]["k"], 0.05, "LDH", 25, 2,
                                    adaptive=params[i]["adaptive_eps"])
        assert np.array_equal(parts[i], ref) and sts[i] == rst


def _kway_cases(seed, n):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = i % 4
        if kind == 0:
            out.append(synth.c3_instance(900 + i, N=int(rng.integers(800, 20000))))
        elif kind == 1:
            r = int(rng.integers(400, 5000))
            out.append(synth.rownet(r, r, seed=300 + i))
        elif kind == 2:
            out.append(synth.uniform(int(rng.integers(100, 4000)), int(rng.integers(100, 4000)), 2, 9,
                                     seed=400 + i))
        else:  # weighted nodes and hyperedges, duplicate and single pins
            N, E = int(rng.integers(200, 3000)), int(rng.integers(100, 3000))
            deg = rng.integers(0, 12, size=E)
            hoff = np.zeros(E + 1, np.int32)
            hoff[1:] = np.cumsum(deg)
            out.append(dict(N=N, E=E, hoff=hoff, pins=rng.integers(0, N, size=int(hoff[-1])).astype(np.int32),
                            nw=rng.integers(1, 9, size=N).astype(np.int32),
                            hw=rng.integers(1, 50, size=E).astype(np.int32)))
    return out


def test_block_path_kway_matches_oracle_in_one_launch_per_bucket():
    # k > 2 instances run their nested bisections inside the persistent blocks: the batch makes
    # at most one launch per size bucket (no worker-pool fallback), and every result equals the
    # oracle's Algorithm 6
    import paper_2012_13618_gb300 as bp
    graphs = _kway_cases(21, 36)
    ks = [3, 4, 5, 8, 16, 64, 7, 2, 1, 33, 12, 6]
    pols = ["LDH", "HDH", "LWD", "HWD", "RAND"]
    params = [dict(k=ks[i % len(ks)], eps=[0.05, 0.1, 0.0][i % 3], policy=pols[i % 5], levels=[25, 4, 25][i % 3],
                   iters=[2, 1, 3][i % 3], adaptive_eps=bool(i % 2)) for i in range(len(graphs))]
    before = bp.kernel_launches()
    parts, st = bp.partition_batch(graphs, params, workers=2)
    assert bp.kernel_launches() - before <= 4
    for i, g in enumerate(graphs):
        p = params[i]
        ref, rst = oracle.partition(oracle.Hypergraph.from_dict(g), p["k"], p["eps"], p["policy"], p["levels"],
                                    p["iters"], adaptive=p["adaptive_eps"])
        assert np.array_equal(parts[i], ref), (i, p)
        assert st[i] == rst, (i, p)


def test_block_graph_replayed_on_new_data_of_the_same_shape():
    # a second batch with the same sizes and parameters replays the captured graph; its inputs are
    # new (pins permuted within every hyperedge's node set), so a stale copy would show
    import paper_2012_13618_gb300 as bp
    rng = np.random.default_rng(33)
    a = [synth.uniform(int(n), int(n) + 50, 2, 7, seed=500 + i) for i, n in enumerate(rng.integers(500, 6000, 10))]
    b = []
    for i, g in enumerate(a):
        perm = np.random.default_rng(600 + i).permutation(g["N"]).astype(np.int32)
        b.append(dict(g, pins=perm[g["pins"]]))
    params = [dict(k=[2, 4, 8][i % 3], eps=0.05, policy="LDH", levels=25, iters=2) for i in range(10)]
    for graphs in (a, b, a):
        before = bp.kernel_launches()
        parts, st = bp.partition_batch(graphs, params, workers=2)
        launched = bp.kernel_launches() - before
        for i, g in enumerate(graphs):
            ref, rst = oracle.partition(oracle.Hypergraph.from_dict(g), params[i]["k"], 0.05, "LDH", 25, 2)
            assert np.array_equal(parts[i], ref) and st[i] == rst, i
    assert launched == 0  # the third call replayed the graph captured by the first


def test_tuner_writes_cache_and_results_stay_exact(tmp_path, monkeypatch):
    import json
    import paper_2012_13618_gb300 as bp
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("BIPART_TUNE_CACHE", str(cache))
    graphs = _kway_cases(44, 16) + [synth.c3_instance(970, N=30000)]
    params = [dict(k=[2, 4][i % 2], eps=0.05, policy="LDH", levels=25, iters=2) for i in range(len(graphs))]
    chosen = bp.tune_batch(graphs, params)
    assert chosen and all((t, m) in ((256, 1), (256, 2), (256, 4), (512, 1), (512, 2), (1024, 1))
                          for t, m in chosen.values())
    doc = json.loads(cache.read_text())
    assert doc["version"] == 1 and len(doc["devices"]) == 1
    (entry,) = doc["devices"].values()
    stored = {int(b): tuple(v) for b, v in entry.items()}
    assert all(stored[b] == v for b, v in chosen.items())
    parts, st = bp.partition_batch(graphs, params, workers=2)
    for i, g in enumerate(graphs):
        ref, rst = oracle.partition(oracle.Hypergraph.from_dict(g), params[i]["k"], 0.05, "LDH", 25, 2)
        assert np.array_equal(parts[i], ref) and st[i] == rst, i


def test_server_micro_batches_a_backlog_exactly():
    # many small requests submitted at once leave a backlog, which free workers take as
    # micro-batches through the persistent block path; every result equals the oracle's
    import paper_2012_13618_gb300 as bp
    graphs = mixed_instances(48, seed=12)
    ks = [2, 4, 16, 3]
    refs = [oracle.partition(oracle.Hypergraph.from_dict(g), ks[i % 4], 0.05, "LDH", 25, 2)
            for i, g in enumerate(graphs)]
    with bp.Server(hbm_budget_bytes=0, workers=2) as srv:
        tickets = [srv.submit(g, k=ks[i % 4], eps=0.05) for i, g in enumerate(graphs)]
        for i, t in enumerate(tickets):
            parts, st, qms, rms = srv.wait(t)
            assert np.array_equal(parts, refs[i][0]) and st == refs[i][1], i
            assert qms >= 0 and rms >= 0
        batches, batched = srv.stats()
    assert batches >= 1 and batched >= 8


def test_refine_kept_equals_full_bisections():
    # Algorithm 3 and the refinement re-run on a kept hierarchy give what a full bisection with
    # the new imbalance and iteration count gives: with the cluster tail starting partway down
    # (netlist) and from level 0 (small uniform hypergraph)
    import paper_2012_13618_gb300 as bp
    cases = [(synth.c1_netlist(N=100_000), "LDH", 25), (synth.uniform(3000, 3500, 2, 7, seed=71), "RAND", 3)]
    for g, pol, lev in cases:
        hr = oracle.Hypergraph.from_dict(g)
        with bp.create_from(g) as h:
            h.partition(2, 0.05, pol, lev, 2)
            for eps, it in ((0.05, 0), (0.05, 4), (0.1, 1), (0.0, 2)):
                parts, st = h.refine_kept(eps, it)
                ref = oracle.bisect(hr, eps, pol, lev, it, keep_levels=False)
                assert np.array_equal(parts, ref["side"].astype(np.int32)), (pol, eps, it)
                assert st == ref["status"], (pol, eps, it)
            # the handle's full path is unaffected (its plan is captured and replayed afterwards)
            for _ in range(3):
                parts, st = h.partition(2, 0.1, pol, lev, 1)
            ref = oracle.bisect(hr, 0.1, pol, lev, 1, keep_levels=False)
            assert np.array_equal(parts, ref["side"].astype(np.int32))
            h.partition(4, 0.05, pol, lev, 2)
            with pytest.raises(bp.BipartError):
                h.refine_kept(0.05, 2)


def test_batch_release_then_reuse():
    # the buffers, arenas, graph and pool the batch call keeps are freed, and the next call
    # builds them again with the same results
    import paper_2012_13618_gb300 as bp
    graphs = mixed_instances(8, seed=77)
    params = [dict(k=[2, 4][i % 2], eps=0.05, policy="LDH", levels=25, iters=2) for i in range(len(graphs))]
    a, sa = bp.partition_batch(graphs, params, workers=2)
    bp.batch_release()
    b, sb = bp.partition_batch(graphs, params, workers=2)
    assert np.array_equal(sa, sb)
    for x, y, g, p in zip(a, b, graphs, params):
        ref, _ = oracle.partition(oracle.Hypergraph.from_dict(g), p["k"], 0.05, "LDH", 25, 2)
        assert np.array_equal(x, ref) and np.array_equal(y, ref)
