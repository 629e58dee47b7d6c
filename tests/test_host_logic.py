"""Host-side helpers that need no GPU: the Pareto frontier of the design-space sweep and the
marshalling of partition parameters into the C ABI's struct."""
import ctypes

import numpy as np

import paper_2012_13618_gb300 as bp
from paper_2012_13618_gb300.sweep import pareto


def test_pareto_example():
    assert pareto([(1, 5), (2, 3), (3, 4), (2, 3), (0.5, 9)]) == [0, 1, 3, 4]


def test_pareto_against_brute_force():
    rng = np.random.default_rng(8)
    for _ in range(200):
        n = int(rng.integers(1, 12))
        pts = [(int(rng.integers(0, 6)), int(rng.integers(0, 6))) for _ in range(n)]
        front = set(pareto(pts))
        for i, (ti, ci) in enumerate(pts):
            better = [j for j, (tj, cj) in enumerate(pts)
                      if tj <= ti and cj <= ci and (tj < ti or cj < ci)]
            assert (i in front) == (not better), (pts, i)


def test_params_marshalling():
    p = bp._params(6, 0.05, "HWD", 7, 3, adaptive_eps=True, merge_parallel=True)
    assert (p.k, p.policy, p.levels, p.refine_iters) == (6, bp.POLICIES["HWD"], 7, 3)
    assert abs(p.epsilon - 0.05) < 1e-15
    assert p.flags == bp.FLAG_ADAPTIVE_EPS | bp.FLAG_MERGE_PARALLEL
    assert bp._params().flags == 0
    # the struct matches the header's layout: int32 k; double epsilon; 4 x int32
    assert ctypes.sizeof(bp.Params) == 32


def test_roofline_traffic_record_tracks_the_sources(monkeypatch, tmp_path):
    # the DRAM traffic bench.py reports comes from an ncu record in profiles/ only while the
    # record's source hash matches the kernel's current sources; it scales with the launch
    import json
    import bench
    (tmp_path / "profiles").mkdir()
    rec = {"kernel": "node_gain", "dram_bytes": 1000, "source_sha256": "abc"}
    (tmp_path / "profiles" / "node_gain_c1_netlist_1M.md").write_text(
        "# summary\n\ntraffic-record: " + json.dumps(rec) + "\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda name: "abc")
    assert bench.ncu_traffic("node_gain", 50, 100) == 500
    monkeypatch.setattr(bench, "source_hash", lambda name: "def")
    assert bench.ncu_traffic("node_gain", 50, 100) is None
    assert bench.ncu_traffic("no_such_kernel", 50, 100) is None
