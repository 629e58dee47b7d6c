"""Pins of the parallel-net merging switch (reading M1, off by default: the paper never merges
hyperedges).  With it, the coarse hyperedges of a contracted level that have the same sorted pin
list become the one with the smallest id, carrying the sum of their weights."""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _lists(d):
    hoff, pins = d["hoff"], d["pins"]
    return [tuple(pins[hoff[e]:hoff[e + 1]].tolist()) for e in range(len(hoff) - 1)]


def _first_occurrence_grouping(d):
    """The definition written out: walk the hyperedges in id order, keep the first of every
    distinct list, add each later copy's weight to it."""
    keep, weight, where = [], [], {}
    for e, lst in enumerate(_lists(d)):
        if lst in where:
            weight[where[lst]] += int(d["hw"][e])
        else:
            where[lst] = len(keep)
            keep.append(lst)
            weight.append(int(d["hw"][e]))
    return keep, weight


def _with_parallel_nets(seed):
    rng = np.random.default_rng(seed)
    g = synth.uniform(400, 300, 2, 5, seed=seed)
    lists = _lists(dict(hoff=np.asarray(g["hoff"]), pins=np.asarray(g["pins"])))
    # plant copies of some nets (pins shuffled: normalisation sorts them) with random weights
    for _ in range(200):
        lst = list(lists[int(rng.integers(0, len(lists)))])
        rng.shuffle(lst)
        lists.append(tuple(lst))
    order = rng.permutation(len(lists))
    lists = [lists[i] for i in order]
    hoff = np.concatenate([[0], np.cumsum([len(x) for x in lists])]).astype(np.int32)
    pins = np.concatenate([np.asarray(x, np.int32) for x in lists])
    hw = rng.integers(1, 9, size=len(lists)).astype(np.int32)
    return dict(N=g["N"], hoff=hoff, pins=pins, hw=hw)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_merge_is_first_occurrence_grouping(seed):
    h = oracle.Hypergraph.from_dict(_with_parallel_nets(seed))
    before = h.arrays()
    m = oracle.merge_parallel(h).arrays()
    keep, weight = _first_occurrence_grouping(before)
    assert _lists(m) == keep
    assert m["hw"].tolist() == weight
    assert len(set(_lists(m))) == len(_lists(m))          # no parallel nets left
    assert int(m["hw"].sum()) == int(before["hw"].sum())  # total weight conserved


@pytest.mark.parametrize("seed", [1, 2])
def test_merge_preserves_every_cut(seed, rng):
    h = oracle.Hypergraph.from_dict(_with_parallel_nets(seed))
    m = oracle.merge_parallel(h)
    for _ in range(20):
        side = rng.integers(0, 2, size=h.N).astype(np.uint8)
        assert oracle.cut_bisection(h, side) == oracle.cut_bisection(m, side)
        part = rng.integers(0, 5, size=h.N).astype(np.int32)
        assert oracle.cut(h, part) == oracle.cut(m, part)


@pytest.mark.parametrize("policy", ["LDH", "LWD", "HWD", "RAND"])
def test_coarsen_merge_is_coarsen_then_merge(policy):
    g = synth.c1_netlist(N=20_000)
    h = oracle.Hypergraph.from_dict(g)
    c0, cm0, mt0 = oracle.coarsen(h, policy)
    c1, cm1, mt1 = oracle.coarsen_merge(h, policy)
    # merging happens after contraction: the matching and the node map are those of Algorithm 2
    assert np.array_equal(cm0, cm1) and np.array_equal(mt0, mt1)
    keep, weight = _first_occurrence_grouping(c0.arrays())
    assert _lists(c1.arrays()) == keep and c1.arrays()["hw"].tolist() == weight


def test_merge_makes_weight_policies_differ():
    # with unit input weights and no merging, LWD / HWD tie everywhere (reading C5); merged
    # parallel nets give coarse hyperedges real weights, and the two policies part ways
    h = oracle.Hypergraph.from_dict(synth.c1_netlist(N=20_000))
    a = oracle.bisect(h, 0.05, "LWD", 25, 2, keep_levels=False, merge=True)
    b = oracle.bisect(h, 0.05, "HWD", 25, 2, keep_levels=False, merge=True)
    assert not np.array_equal(a["side"], b["side"])


def test_merge_off_is_the_paper():
    h = oracle.Hypergraph.from_dict(synth.uniform(1500, 1600, 2, 6, seed=21))
    for k in (2, 3, 4):
        assert np.array_equal(oracle.partition(h, k)[0], oracle.partition(h, k, merge=False)[0])
    r0 = oracle.bisect(h, 0.1, "LDH", 25, 2, keep_levels=False)
    r1 = oracle.bisect(h, 0.1, "LDH", 25, 2, keep_levels=False, e6=100_000)
    assert np.array_equal(r0["side"], r1["side"])
