"""The cluster tail (the coarse levels of a bisection in one thread-block-cluster launch) against
the oracle when it starts from large levels, where its chunk streaming, wide chunks and block-tier
contraction all run, and the grid path alone with the tail switched off.  The start limits are
read once per process, so the partitions run in child processes with the limits overridden; the
oracle runs here.  Integer arithmetic: the partition and the status must be identical."""
import json
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import torch, synth, paper_2012_13618_gb300 as bp
torch.cuda.set_device(0)
bp.use_torch_allocator()
spec = json.loads(sys.argv[2])
out = {}
for name, gen, k, eps, policy, levels, iters in spec:
    g = eval(gen, {"synth": synth, "np": np})
    with bp.create_from(g) as h:
        runs = [h.partition(k, eps, policy, levels, iters) for _ in range(3)]
        nlev = h.num_levels() if k == 2 else -1
    out[name] = [[r[0].tolist(), int(r[1])] for r in runs] + [nlev]
json.dump(out, open(sys.argv[3], "w"))
"""


def weighted_graph(seed, N, E, dmax):
    rng = np.random.default_rng(seed)
    deg = rng.integers(0, dmax + 1, size=E)
    deg[:3] = 400  # hyperedges wide enough for the warp and block tiers
    hoff = np.zeros(E + 1, np.int32)
    hoff[1:] = np.cumsum(deg)
    pins = rng.integers(0, N, size=int(hoff[-1])).astype(np.int32)
    return dict(N=N, E=E, hoff=hoff, pins=pins, nw=rng.integers(1, 6, size=N).astype(np.int32),
                hw=rng.integers(1, 9, size=E).astype(np.int32))


CASES = [
    ("netlist_1m", "synth.c1_netlist()", 2, 0.05, "LDH", 25, 2),
    ("netlist_200k_hdh", "synth.c1_netlist(N=200_000)", 2, 0.05, "HDH", 25, 2),
    ("rownet_300k", "synth.rownet(300_000, 300_000, seed=2)", 2, 0.05, "LDH", 25, 2),
    ("uniform_12k_rand", "synth.uniform(12_000, 30_000, 2, 9, seed=5)", 2, 0.1, "RAND", 25, 3),
    ("netlist_100k_k4", "synth.c1_netlist(N=100_000)", 4, 0.05, "LDH", 25, 2),
]


def _graph(gen):
    return eval(gen, {"synth": synth, "np": np})


def _run_child(env_over, cases):
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "out.json")
        env = dict(os.environ, **env_over)
        subprocess.run([sys.executable, "-c", CHILD, ROOT, json.dumps(cases), out], env=env, check=True,
                       timeout=600)
        return json.load(open(out))


def _check(res, cases):
    for name, gen, k, eps, policy, levels, iters in cases:
        hr = oracle.Hypergraph.from_dict(_graph(gen))
        if k == 2:
            ref = oracle.bisect(hr, eps, policy, levels, iters, keep_levels=False)
            want, wst = ref["side"].astype(np.int32), ref["status"]
            assert res[name][-1] == ref["nlev"], name
        else:
            want, wst = oracle.partition(hr, k, eps, policy, levels, iters)
        for parts, st in res[name][:-1]:
            assert np.array_equal(np.asarray(parts, np.int32), want) and st == wst, name


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")


def test_tail_from_large_levels_matches_oracle():
    # the tail takes every level of <= 12,288 nodes whatever its pins (up to 4M)
    _check(_run_child({"BIPART_TAIL_PINS": "4000000"}, CASES), CASES)


def test_weighted_tail_with_wide_hyperedges_matches_oracle():
    cases = [("weighted_%d" % s, "None", 2, 0.05, pol, 25, 2) for s, pol in ((1, "LDH"), (2, "LWD"), (3, "HWD"))]
    graphs = {c[0]: weighted_graph(10 + i, 9000, 20000, 12) for i, c in enumerate(cases)}
    with tempfile.TemporaryDirectory() as d:
        specs = []
        for c in cases:
            path = os.path.join(d, c[0] + ".npz")
            g = graphs[c[0]]
            np.savez(path, hoff=g["hoff"], pins=g["pins"], nw=g["nw"], hw=g["hw"])
            gen = ("(lambda z: dict(N=9000, E=20000, hoff=z['hoff'], pins=z['pins'], nw=z['nw'], "
                   "hw=z['hw']))(np.load(%r))" % path)
            specs.append((c[0], gen) + c[2:])
        res = _run_child({"BIPART_TAIL_PINS": "4000000"}, specs)
        for c, s in zip(cases, specs):
            hr = oracle.Hypergraph.from_dict(graphs[c[0]])
            ref = oracle.bisect(hr, c[3], c[4], c[5], c[6], keep_levels=False)
            for parts, st in res[c[0]][:-1]:
                assert np.array_equal(np.asarray(parts, np.int32), ref["side"].astype(np.int32)), c[0]
                assert st == ref["status"], c[0]


def test_grid_path_alone_matches_oracle():
    # the tail switched off: every level on the grid path
    cases = [c for c in CASES if c[0] in ("netlist_200k_hdh", "uniform_12k_rand")]
    _check(_run_child({"BIPART_TAIL_NODES": "0"}, cases), cases)
