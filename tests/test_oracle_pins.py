"""Pins of the CPU oracle against what the paper and mathematics fix (no GPU).

Each test names the passage it follows.  Hand-derived worked examples live in tests/golden/
(each with its citation and derivation); the rest are closed forms, brute force on tiny inputs,
identities and invariants chosen so that a dropped term, a flipped sign or a transposed operand
in the oracle fails at least one of them.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def path_graph(n):
    hoff = np.arange(0, 2 * (n - 1) + 1, 2, dtype=np.int32)
    pins = np.array([x for i in range(n - 1) for x in (i, i + 1)], dtype=np.int32)
    return hoff, pins


def random_hg(rng, N, E, dmax=5, weights=False, hweights=False, dup=False):
    deg = rng.integers(1, dmax + 1, size=E)
    hoff = np.zeros(E + 1, np.int32)
    hoff[1:] = np.cumsum(deg)
    if dup:
        pins = rng.integers(0, N, size=int(hoff[-1])).astype(np.int32)
    else:
        pins = np.concatenate([rng.choice(N, size=min(d, N), replace=False) for d in deg]
                              ).astype(np.int32) if E else np.zeros(0, np.int32)
        hoff[1:] = np.cumsum(np.minimum(deg, N))
    nw = rng.integers(1, 5, size=N).astype(np.int32) if weights else None
    hw = rng.integers(1, 4, size=E).astype(np.int32) if hweights else None
    return N, hoff, pins, nw, hw


def lam_cut_direct(h, part):
    a = h.arrays()
    return sum(int(a["hw"][e]) * (len(set(part[a["pins"][a["hoff"][e]:a["hoff"][e + 1]]])) - 1)
               for e in range(a["E"]))


# ----------------------------------------------------------------------------- hash (reading C1)
def test_hash_published_vectors():
    g = gold("murmur3_fmix32.json")
    for x, y in g["cases"]:
        assert oracle.hash32(x) == y


def _inv_xorshift_right(y, s):
    x = y
    for _ in range(32 // s + 1):
        x = y ^ (x >> s)
    return x & 0xFFFFFFFF


def test_hash_is_a_bijection(rng):
    # Invert the finaliser step by step (xorshift inverse, modular inverse of the odd
    # multipliers): a round trip on random inputs shows (priority, hash) is unique per id.
    m1, m2 = 0x85EBCA6B, 0xC2B2AE35
    i1, i2 = pow(m1, -1, 2**32), pow(m2, -1, 2**32)
    for x in rng.integers(0, 2**32, size=2000, dtype=np.uint64).tolist():
        y = oracle.hash32(x)
        y = _inv_xorshift_right(y, 16)
        y = (y * i2) & 0xFFFFFFFF
        y = _inv_xorshift_right(y, 13)
        y = (y * i1) & 0xFFFFFFFF
        y = _inv_xorshift_right(y, 16)
        assert y == x


# ----------------------------------------------------------------------------- small closed forms
def test_ceil_sqrt():
    for n in list(range(0, 2000)) + [10**6, 10**6 + 1, 5 * 10**6, 2**31 - 1]:
        want = 0 if n == 0 else math.isqrt(n - 1) + 1
        assert oracle.ceil_sqrt(n) == want


@pytest.mark.parametrize("W,eps,want", [(10000, 0.1, 5500), (9, 0.0, 5), (11, 0.0, 6),
                                        (2500588, 0.05, 1312808), (1, 0.1, 1), (0, 0.1, 0),
                                        (100, 0.001, 50), (101, 0.01, 51)])
def test_balance_limit(W, eps, want):
    # Sec. 1.1: |V_i| <= (1 + eps) |V| / k with k = 2, floored, never below ceil(W/2) (C12).
    assert oracle.limit(W, eps) == want


def test_normalise_definition(rng):
    # Reading C10: sorted unique pins, hyperedges with < 2 distinct pins dropped, order kept.
    for _ in range(20):
        N, hoff, pins, nw, hw = random_hg(rng, 12, 15, dmax=6, hweights=True, dup=True)
        h = oracle.Hypergraph.from_csr(N, hoff, pins, nw, hw)
        a = h.arrays()
        want = [(sorted(set(pins[hoff[e]:hoff[e + 1]].tolist())), int(hw[e]))
                for e in range(len(hoff) - 1)]
        want = [x for x in want if len(x[0]) >= 2]
        got = [(a["pins"][a["hoff"][e]:a["hoff"][e + 1]].tolist(), int(a["hw"][e]))
               for e in range(a["E"])]
        assert got == want


# ----------------------------------------------------------------------------- Algorithm 1
def _brute_match(a, policy):
    """Lexicographic argmin over incident hyperedges of (priority, hash(id), id)."""
    E, N = a["E"], a["N"]
    best = [None] * N
    for e in range(E):
        d = int(a["hoff"][e + 1] - a["hoff"][e])
        w = int(a["hw"][e])
        h = oracle.hash32(e)
        pr = {0: d, 1: 0xFFFFFFFF - d, 2: w, 3: 0xFFFFFFFF - w, 4: h}[policy]
        for v in a["pins"][a["hoff"][e]:a["hoff"][e + 1]].tolist():
            key = (pr, h, e)
            if best[v] is None or key < best[v]:
                best[v] = key
    return np.array([-1 if b is None else b[2] for b in best], np.int32)


@pytest.mark.parametrize("policy", [0, 1, 2, 3, 4])
def test_match_is_lexicographic_argmin(rng, policy):
    for _ in range(15):
        N, hoff, pins, nw, hw = random_hg(rng, 25, 18, dmax=5, hweights=True)
        h = oracle.Hypergraph.from_csr(N, hoff, pins, nw, hw)
        a = h.arrays()
        assert np.array_equal(oracle.match(h, policy), _brute_match(a, policy))


def test_match_literal_three_passes(rng):
    # Algorithm 1 as printed (third pass tests rand only) equals the oracle's matching.
    for _ in range(10):
        N, hoff, pins, _, _ = random_hg(rng, 30, 25, dmax=4)
        h = oracle.Hypergraph.from_csr(N, hoff, pins)
        a = h.arrays()
        pri = [math.inf] * N
        rnd = [math.inf] * N
        hid = [math.inf] * N
        edges = [(e, a["pins"][a["hoff"][e]:a["hoff"][e + 1]].tolist()) for e in range(a["E"])]
        for e, ps in edges:
            for v in ps:
                pri[v] = min(pri[v], len(ps))
        for e, ps in edges:
            for v in ps:
                if len(ps) == pri[v]:
                    rnd[v] = min(rnd[v], oracle.hash32(e))
        for e, ps in edges:
            for v in ps:
                if oracle.hash32(e) == rnd[v]:
                    hid[v] = min(hid[v], e)
        want = np.array([-1 if x == math.inf else x for x in hid], np.int32)
        assert np.array_equal(oracle.match(h, "LDH"), want)


def test_graph_ldh_matching_by_hand():
    # Graph special case: all degrees 2, so LDH reduces to the smallest hash among incident edges.
    # Path 0-1-2-3: edge ids 0,1,2 hash to 0, 0x514e28b7, 0x30f4c306 (published-vector pinned).
    hoff, pins = path_graph(4)
    h = oracle.Hypergraph.from_csr(4, hoff, pins)
    # node 0: edge 0; node 1: edges 0,1 -> 0; node 2: edges 1,2 -> hash(2) < hash(1) -> 2; node 3: 2
    assert oracle.match(h, "LDH").tolist() == [0, 0, 2, 2]


# ----------------------------------------------------------------------------- Algorithm 2
def test_fig2_constructed():
    g = gold("fig2_constructed.json")
    h = oracle.Hypergraph.from_csr(g["N"], g["hoff"], g["pins"])
    c, cmap, m = oracle.coarsen(h, g["policy"])
    a = c.arrays()
    assert m.tolist() == g["match"]
    assert cmap.tolist() == g["cmap"]
    assert a["hoff"].tolist() == g["coarse_hoff"]
    assert a["pins"].tolist() == g["coarse_pins"]
    assert a["nw"].tolist() == g["coarse_nw"]


def test_singleton_attach_constructed():
    g = gold("singleton_attach.json")
    for case in g["cases"]:
        h = oracle.Hypergraph.from_csr(g["N"], g["hoff"], g["pins"], case["nw"])
        c, cmap, _ = oracle.coarsen(h, "LDH")
        a = c.arrays()
        assert cmap.tolist() == case["cmap"]
        assert a["nw"].tolist() == case["coarse_nw"]
        assert a["hoff"].tolist() == case["coarse_hoff"]
        assert a["pins"].tolist() == case["coarse_pins"]


def check_coarsen_properties(a, c, cmap, m):
    """Properties of Algorithm 2 (readings C6-C9) that determine cmap uniquely from the matching."""
    N, E = a["N"], a["E"]
    nw = a["nw"]
    S = {}
    for v in range(N):
        if m[v] >= 0:
            S.setdefault(int(m[v]), []).append(v)
    merged_group = {v: e for e, vs in S.items() if len(vs) > 1 for v in vs}
    gw = {e: sum(int(nw[v]) for v in vs) for e, vs in S.items() if len(vs) > 1}
    # expected final group of every node
    grp = {}
    for v in range(N):
        if v in merged_group:
            grp[v] = ("g", merged_group[v])
        elif m[v] >= 0:
            e = int(m[v])
            cands = [merged_group[u] for u in a["pins"][a["hoff"][e]:a["hoff"][e + 1]].tolist()
                     if u in merged_group]
            grp[v] = ("g", min(cands, key=lambda x: (gw[x], x))) if cands else ("s", v)
        else:
            grp[v] = ("s", v)
    members = {}
    for v in range(N):
        members.setdefault(grp[v], []).append(v)
    order = sorted(members.values(), key=min)
    want = np.empty(N, np.int32)
    for cid, vs in enumerate(order):
        want[vs] = cid
    assert np.array_equal(cmap, want)
    # every merged set lies inside one fine hyperedge (its matched hyperedge)
    for e, vs in S.items():
        pe = set(a["pins"][a["hoff"][e]:a["hoff"][e + 1]].tolist())
        assert set(vs) <= pe
    # weights conserved, coarse hyperedges are the contracted fine ones with >= 2 parents
    b = c.arrays()
    assert b["nw"].sum() == nw.sum()
    assert np.array_equal(np.bincount(cmap, weights=nw, minlength=b["N"]).astype(np.int64),
                          b["nw"].astype(np.int64))
    exp = []
    for e in range(E):
        ps = sorted(set(cmap[a["pins"][a["hoff"][e]:a["hoff"][e + 1]]].tolist()))
        if len(ps) >= 2:
            exp.append((ps, int(a["hw"][e])))
    got = [(b["pins"][b["hoff"][e]:b["hoff"][e + 1]].tolist(), int(b["hw"][e]))
           for e in range(b["E"])]
    assert got == exp
    assert b["N"] <= N


@pytest.mark.parametrize("policy", [0, 1, 2, 3, 4])
def test_coarsen_properties_random(rng, policy):
    for _ in range(12):
        N, hoff, pins, nw, hw = random_hg(rng, 40, 30, dmax=6, weights=True, hweights=True)
        h = oracle.Hypergraph.from_csr(N, hoff, pins, nw, hw)
        c, cmap, m = oracle.coarsen(h, policy)
        check_coarsen_properties(h.arrays(), c, cmap, m)


def test_coarsen_every_level_c0():
    h = oracle.Hypergraph.from_dict(synth.uniform(600, 600, 2, 6, seed=7))
    r = oracle.bisect(h, 0.1, "LDH", 25, 2)
    for l in range(r["nlev"] - 1):
        a = r["levels"][l]
        b = oracle.Hypergraph.from_csr(a["N"], a["hoff"], a["pins"], a["nw"], a["hw"])
        c, cmap, m = oracle.coarsen(b, "LDH")
        assert np.array_equal(cmap, r["cmaps"][l])
        check_coarsen_properties(a, c, cmap, m)
        assert np.array_equal(c.arrays()["pins"], r["levels"][l + 1]["pins"])


def test_one_hyperedge_collapses():
    n = 17
    h = oracle.Hypergraph.from_csr(n, [0, n], np.arange(n))
    c, cmap, _ = oracle.coarsen(h, "LDH")
    assert c.N == 1 and c.E == 0 and cmap.tolist() == [0] * n


def test_disjoint_hyperedges_collapse():
    # pairwise-disjoint hyperedges over nodes 0..11, nodes 12..14 isolated
    hoff = [0, 3, 5, 9, 12]
    pins = [0, 4, 8, 1, 2, 3, 5, 6, 7, 9, 10, 11]
    h = oracle.Hypergraph.from_csr(15, hoff, pins)
    c, cmap, m = oracle.coarsen(h, "RAND")
    assert c.N == 4 + 3 and c.E == 0
    assert m[12:].tolist() == [-1, -1, -1]
    # groups numbered by smallest member: {0,4,8}->0, {1,2}->1, {3,5,6,7}->2, {9,10,11}->3
    assert cmap.tolist() == [0, 1, 1, 2, 0, 2, 2, 2, 0, 3, 3, 3, 4, 5, 6]


def test_projection_preserves_cut(rng):
    h = oracle.Hypergraph.from_dict(synth.uniform(800, 900, 2, 6, seed=3))
    r = oracle.bisect(h, 0.1, "HDH", 25, 2)
    for l in range(r["nlev"] - 1):
        fine = r["levels"][l]
        coarse = r["levels"][l + 1]
        hf = oracle.Hypergraph.from_csr(fine["N"], fine["hoff"], fine["pins"], fine["nw"], fine["hw"])
        hc = oracle.Hypergraph.from_csr(coarse["N"], coarse["hoff"], coarse["pins"], coarse["nw"],
                                        coarse["hw"])
        for k in (2, 3):
            pc = rng.integers(0, k, size=coarse["N"]).astype(np.int32)
            assert oracle.cut(hc, pc) == oracle.cut(hf, pc[r["cmaps"][l]])


# ----------------------------------------------------------------------------- cut and gains
def test_cut_by_hand():
    # hyperedges {0,1,2} w=2, {2,3} w=1, {0,3,4} w=5 with parts [0,0,1,1,2]
    h = oracle.Hypergraph.from_csr(5, [0, 3, 5, 8], [0, 1, 2, 2, 3, 0, 3, 4], None, [2, 1, 5])
    assert oracle.cut(h, np.array([0, 0, 1, 1, 2])) == 2 * 1 + 1 * 0 + 5 * 2
    assert oracle.cut_bisection(h, np.array([0, 0, 1, 1, 1])) == 2 + 5


def test_cut_two_ways(rng):
    for _ in range(20):
        N, hoff, pins, nw, hw = random_hg(rng, 30, 40, dmax=7, hweights=True)
        h = oracle.Hypergraph.from_csr(N, hoff, pins, nw, hw)
        side = rng.integers(0, 2, size=N).astype(np.uint8)
        assert oracle.cut(h, side.astype(np.int32)) == oracle.cut_bisection(h, side)
        part = rng.integers(0, 4, size=N).astype(np.int32)
        assert oracle.cut(h, part) == lam_cut_direct(h, part)


def test_gain_equals_bruteforce_cut_delta(rng):
    # Algorithm 4: gain(u) = cut before - cut after moving u alone.
    for _ in range(20):
        N, hoff, pins, nw, hw = random_hg(rng, 60, 70, dmax=6, weights=True, hweights=True)
        h = oracle.Hypergraph.from_csr(N, hoff, pins, nw, hw)
        side = rng.integers(0, 2, size=N).astype(np.uint8)
        g = oracle.gains(h, side)
        base = oracle.cut_bisection(h, side)
        for u in range(N):
            s2 = side.copy()
            s2[u] ^= 1
            assert g[u] == base - oracle.cut_bisection(h, s2), u


# ----------------------------------------------------------------------------- Algorithms 3 and 5
def test_initial_path9():
    g = gold("path9_initial.json")
    hoff, pins = path_graph(g["N"])
    h = oracle.Hypergraph.from_csr(g["N"], hoff, pins)
    side, rounds = oracle.initial(h)
    assert side.tolist() == g["side"] and rounds == g["rounds"]


def test_initial_without_hyperedges():
    # E = 0: all gains are 0, so nodes move in ascending id, s at a time, until W0 >= W1.
    for n in (1, 2, 4, 7, 16, 36, 50, 101):
        h = oracle.Hypergraph.from_csr(n, [0], [])
        side, rounds = oracle.initial(h)
        s = oracle.ceil_sqrt(n)
        r = 0
        while r * s < n and 2 * min(r * s, n) < n:
            r += 1
        moved = min(r * s, n)
        assert rounds == r
        assert side.tolist() == [0] * moved + [1] * (n - moved)


def test_initial_against_bruteforce_gains(rng):
    # Algorithm 3 on random weighted hypergraphs, replayed with brute-force single-move gains:
    # while side 0 holds less than half the weight, the ceil(sqrt n) nodes of side 1 with the
    # largest gain (smaller id first) move to side 0 (reading C14)
    for _ in range(25):
        N, hoff, pins, nw, hw = random_hg(rng, 36, 40, dmax=5, weights=True, hweights=True)
        h = oracle.Hypergraph.from_csr(N, hoff, pins, nw, hw)
        w = np.asarray(h.arrays()["nw"], np.int64)
        W = int(w.sum())
        s = oracle.ceil_sqrt(N)
        side = np.ones(N, np.uint8)
        rounds = 0
        while 2 * int(w[side == 0].sum()) < W:
            rounds += 1
            base = oracle.cut_bisection(h, side)
            gain = {}
            for u in np.nonzero(side == 1)[0]:
                s2 = side.copy()
                s2[u] = 0
                gain[int(u)] = base - oracle.cut_bisection(h, s2)
            for u in sorted(gain, key=lambda u: (-gain[u], u))[:s]:
                side[u] = 0
        got, got_rounds = oracle.initial(h)
        assert got_rounds == rounds and np.array_equal(got, side)


def test_refine_path9():
    g = gold("path9_refine.json")
    hoff, pins = path_graph(9)
    h = oracle.Hypergraph.from_csr(9, hoff, pins)
    side = np.array(g["side_before"], np.uint8)
    assert oracle.gains(h, side).tolist() == g["gains"]
    assert oracle.cut_bisection(h, side) == g["cut_before"]
    assert oracle.refine_iter(h, side) == g["lmin"]
    assert side.tolist() == g["side_after"]
    assert oracle.cut_bisection(h, side) == g["cut_after"]


def test_refine_iteration_properties(rng):
    # Algorithm 5 on random hypergraphs, checked against brute-force cut deltas: the same number
    # of nodes leaves each side (l_min), every mover had a non-negative single-move gain, and
    # on each side no staying node with gain >= 0 ranks before a mover in (gain desc, id asc)
    for _ in range(30):
        N, hoff, pins, nw, hw = random_hg(rng, 50, 60, dmax=6, weights=True, hweights=True)
        h = oracle.Hypergraph.from_csr(N, hoff, pins, nw, hw)
        before = rng.integers(0, 2, size=N).astype(np.uint8)
        base = oracle.cut_bisection(h, before)
        delta = np.empty(N, np.int64)
        for u in range(N):
            s2 = before.copy()
            s2[u] ^= 1
            delta[u] = base - oracle.cut_bisection(h, s2)
        side = before.copy()
        lmin = oracle.refine_iter(h, side)
        moved = np.nonzero(side != before)[0]
        assert len(moved) == 2 * lmin
        for s in (0, 1):
            movers = [u for u in moved if before[u] == s]
            assert len(movers) == lmin
            assert all(delta[u] >= 0 for u in movers)
            stayers = [u for u in range(N) if before[u] == s and side[u] == s and delta[u] >= 0]
            if movers:
                worst = max(movers, key=lambda u: (-delta[u], u))
                assert all((-delta[v], v) > (-delta[worst], worst) for v in stayers)
            cand = sum(1 for u in range(N) if before[u] == s and delta[u] >= 0)
            assert lmin <= cand
        assert lmin == min(sum(1 for u in range(N) if before[u] == t and delta[u] >= 0) for t in (0, 1))


def test_rebalance_path9():
    g = gold("path9_rebalance.json")
    hoff, pins = path_graph(9)
    h = oracle.Hypergraph.from_csr(9, hoff, pins)
    assert oracle.limit(9, g["eps"]) == g["limit"]
    side = np.array(g["side_before"], np.uint8)
    st, rounds = oracle.rebalance(h, side, g["limit"])
    assert (st, rounds) == (g["status"], g["rounds"])
    assert side.tolist() == g["side_after"]


def test_rebalance_outcome_properties(rng):
    for _ in range(40):
        N, hoff, pins, nw, hw = random_hg(rng, 50, 60, dmax=5, weights=True)
        h = oracle.Hypergraph.from_csr(N, hoff, pins, nw, hw)
        w = h.arrays()["nw"]
        side = (rng.random(N) < rng.random()).astype(np.uint8)
        lim = oracle.limit(int(w.sum()), float(rng.choice([0.0, 0.05, 0.2])))
        st, _ = oracle.rebalance(h, side, lim)
        W = [int(w[side == 0].sum()), int(w[side == 1].sum())]
        if st == oracle.OK:
            assert max(W) <= lim
        else:
            H = 0 if W[0] > lim else 1
            assert W[H] > lim
            assert not np.any(w[side == H] <= lim - W[1 - H])


def test_rebalance_against_bruteforce_gains(rng):
    # reading C13 replayed with brute-force single-move gains: while a side is above the limit,
    # its nodes that fit the other side's room, ordered (gain desc, id asc), move as the shortest
    # prefix reaching the excess, at most ceil(sqrt n) nodes and never past the room
    for _ in range(40):
        N, hoff, pins, nw, hw = random_hg(rng, 36, 40, dmax=5, weights=True, hweights=True)
        h = oracle.Hypergraph.from_csr(N, hoff, pins, nw, hw)
        w = np.asarray(h.arrays()["nw"], np.int64)
        lim = oracle.limit(int(w.sum()), float(rng.choice([0.0, 0.05, 0.2])))
        start = (rng.random(N) < rng.random()).astype(np.uint8)
        side = start.copy()
        s = oracle.ceil_sqrt(N)
        status, rounds = oracle.OK, 0
        while True:
            W = [int(w[side == 0].sum()), int(w[side == 1].sum())]
            H = 0 if W[0] > lim else (1 if W[1] > lim else -1)
            if H < 0:
                break
            room, need = lim - W[1 - H], W[H] - lim
            cand = [int(u) for u in np.nonzero(side == H)[0] if w[u] <= room]
            if not cand:
                status = oracle.WARN_IMBALANCED
                break
            rounds += 1
            base = oracle.cut_bisection(h, side)
            gain = {}
            for u in cand:
                s2 = side.copy()
                s2[u] ^= 1
                gain[u] = base - oracle.cut_bisection(h, s2)
            take, acc = [], 0
            for u in sorted(cand, key=lambda u: (-gain[u], u)):
                if len(take) == s or acc + w[u] > room:
                    break
                take.append(u)
                acc += int(w[u])
                if acc >= need:
                    break
            side[take] = 1 - H
        got = start.copy()
        st, got_rounds = oracle.rebalance(h, got, lim)
        assert (st, got_rounds) == (status, rounds) and np.array_equal(got, side)


# ----------------------------------------------------------------------------- multilevel driver
def test_bisect_levels_zero_runs_on_input():
    h = oracle.Hypergraph.from_dict(synth.uniform(300, 300, 2, 4, seed=5))
    r = oracle.bisect(h, 0.1, "LDH", 0, 2)
    assert r["nlev"] == 1


def test_bisect_stops_when_no_hyperedges():
    # Reading C11: a contraction that leaves N unchanged (only when E = 0) ends coarsening.
    h = oracle.Hypergraph.from_dict(synth.uniform(2000, 1500, 2, 6, seed=9))
    r = oracle.bisect(h, 0.1, "LDH", 25, 2)
    sizes = [(l["N"], l["E"]) for l in r["levels"]]
    assert all(sizes[i + 1][0] < sizes[i][0] for i in range(len(sizes) - 1))
    assert r["nlev"] == 26 or sizes[-1][1] == 0


def test_bisect_path9_golden():
    # Sec. 3.4 on the 9-node path, derived by hand step by step (tests/golden/path9_bisect.json):
    # the driver's order -- Algorithm 3 on the coarsest level, then at every level from the
    # coarsest down: projection (below the coarsest), `iters` Algorithm 5 iterations, rebalance
    g = gold("path9_bisect.json")
    hoff, pins = path_graph(9)
    for c in g["cases"]:
        h = oracle.Hypergraph.from_csr(9, hoff, pins, np.array(c["nw"], np.int32))
        r = oracle.bisect(h, 0.1, "LDH", c["levels"], c["iters"])
        assert r["nlev"] == c["nlev"], c["name"]
        if "cmap0" in c:
            assert r["cmaps"][0].tolist() == c["cmap0"], c["name"]
        assert r["side"].tolist() == c["side"], c["name"]
        assert r["status"] == c["status"], c["name"]
        assert oracle.cut_bisection(h, r["side"]) == c["cut"], c["name"]


def _replay_bisect(h, eps, policy, levels, iters):
    """Sec. 3.4 rebuilt from the oracle's single-step functions in the paper's order: coarsen
    (Algorithm 2) until `levels` contractions or until N stops changing (reading C11); Algorithm 3
    on the coarsest level; then from the coarsest level to the input: project through cmap,
    `iters` Algorithm 5 iterations, the rebalance of reading C13."""
    levs, cmaps = [h], []
    while len(levs) - 1 < levels:
        c, cmap, _ = oracle.coarsen(levs[-1], policy)
        if c.N == levs[-1].N:
            break
        levs.append(c)
        cmaps.append(cmap)
    W = int(np.asarray(h.arrays()["nw"], np.int64).sum())
    lim = oracle.limit(W, eps)
    side, _ = oracle.initial(levs[-1])
    side = np.ascontiguousarray(side, np.uint8)
    status = oracle.OK
    for l in range(len(levs) - 1, -1, -1):
        if l < len(levs) - 1:
            side = np.ascontiguousarray(side[cmaps[l]], np.uint8)
        for _ in range(iters):
            oracle.refine_iter(levs[l], side)
        status, _ = oracle.rebalance(levs[l], side, lim)
    return side, status, len(levs)


def test_bisect_schedule_replayed_from_steps(rng):
    # the driver against its own schedule written out from the single steps, on random weighted
    # hypergraphs, several level counts and iteration counts (a coarsest level left unrefined,
    # a rebalance skipped above level 0, or a projection through the wrong map changes results)
    for trial in range(24):
        N = int(rng.integers(20, 120))
        _, hoff, pins, nw, hw = random_hg(rng, N, int(rng.integers(N // 2, 2 * N)), dmax=5,
                                         weights=True, hweights=bool(trial % 2))
        h = oracle.Hypergraph.from_csr(N, hoff, pins, nw, hw)
        levels = [0, 1, 2, 25][trial % 4]
        iters = [1, 2, 3][trial % 3]
        eps = [0.0, 0.05, 0.1][trial % 3]
        policy = ["LDH", "HDH", "RAND"][trial % 3]
        side, status, nlev = _replay_bisect(h, eps, policy, levels, iters)
        r = oracle.bisect(h, eps, policy, levels, iters, keep_levels=False)
        assert r["nlev"] == nlev and r["status"] == status
        assert np.array_equal(r["side"], side), trial


def _brute_min_cut(a, lim):
    N = a["N"]
    best = None
    w = a["nw"].astype(np.int64)
    assign = (np.arange(2 ** N)[:, None] >> np.arange(N)[None, :]) & 1
    W1 = assign @ w
    ok = (W1 <= lim) & (w.sum() - W1 <= lim)
    cut = np.zeros(2 ** N, np.int64)
    for e in range(a["E"]):
        ps = a["pins"][a["hoff"][e]:a["hoff"][e + 1]]
        s = assign[:, ps].sum(axis=1)
        cut += a["hw"][e] * ((s > 0) & (s < len(ps)))
    if ok.any():
        best = int(cut[ok].min())
    return best


def test_bruteforce_min_cut_small(rng):
    for trial in range(12):
        N = int(rng.integers(6, 15))
        _, hoff, pins, nw, hw = random_hg(rng, N, int(rng.integers(4, 20)), dmax=4)
        h = oracle.Hypergraph.from_csr(N, hoff, pins)
        r = oracle.bisect(h, 0.1, "LDH", 25, 2)
        a = h.arrays()
        opt = _brute_min_cut(a, r["limit"])
        cut = oracle.cut_bisection(h, r["side"])
        W1 = int(r["side"].sum())
        assert opt is not None and cut >= opt
        if r["status"] == oracle.OK:
            assert max(W1, N - W1) <= r["limit"]


def test_two_components_zero_cut_recorded():
    # Two disconnected 8-node cliques-of-pairs: the optimum is 0; BiPart finds it here.
    hoff, pins = [0], []
    for base in (0, 8):
        for i in range(7):
            pins += [base + i, base + i + 1]
            hoff.append(len(pins))
    h = oracle.Hypergraph.from_csr(16, hoff, pins)
    r = oracle.bisect(h, 0.0, "LDH", 25, 2)
    assert _brute_min_cut(h.arrays(), r["limit"]) == 0
    assert oracle.cut_bisection(h, r["side"]) == 0


def test_bisect_deterministic():
    h = oracle.Hypergraph.from_dict(synth.c0_uniform())
    a = oracle.bisect(h, 0.1, "LDH", 25, 2)
    b = oracle.bisect(h, 0.1, "LDH", 25, 2)
    assert np.array_equal(a["side"], b["side"]) and a["nlev"] == b["nlev"]
    for x, y in zip(a["levels"], b["levels"]):
        assert np.array_equal(x["pins"], y["pins"])


# ----------------------------------------------------------------------------- Algorithm 6
@pytest.mark.parametrize("k", [2, 4, 8])
def test_kway_cut_identity(k):
    # Reading C16/C17: the lambda-1 cut of the final parts equals the sum of the cuts of every
    # bisection in the recursion tree, each on its net-split subgraph.
    h = oracle.Hypergraph.from_dict(synth.uniform(1500, 1500, 2, 6, seed=11))
    part, st = oracle.partition(h, k, 0.1, "LDH", 25, 2)
    assert part.min() >= 0 and part.max() < k
    m = k.bit_length() - 1
    total = 0
    for lvl in range(m):
        parts_l = part >> (m - lvl)
        for j in range(2 ** lvl):
            s, l2g = oracle.subgraph(h, parts_l, j)
            side = ((part[l2g] >> (m - lvl - 1)) & 1).astype(np.uint8)
            total += oracle.cut_bisection(s, side)
    assert total == oracle.cut(h, part)


def test_kway_children_equal_solo_bisections():
    h = oracle.Hypergraph.from_dict(synth.uniform(1200, 1300, 2, 5, seed=13))
    part, _ = oracle.partition(h, 4, 0.1, "RAND", 25, 2)
    top = part >> 1
    r = oracle.bisect(h, 0.1, "RAND", 25, 2, keep_levels=False)
    assert np.array_equal(top, r["side"].astype(np.int32))
    for j in (0, 1):
        s, l2g = oracle.subgraph(h, top, j)
        rj = oracle.bisect(s, 0.1, "RAND", 25, 2, keep_levels=False)
        assert np.array_equal(part[l2g] & 1, rj["side"].astype(np.int32))


def _subgraph_restated(a, part, j):
    """Reading C16 written out: the nodes of part j in ascending id, renumbered 0..n-1; every
    hyperedge restricted to them, kept when at least 2 pins remain, in ascending hyperedge id;
    node and hyperedge weights carried."""
    l2g = [v for v in range(a["N"]) if part[v] == j]
    loc = {v: i for i, v in enumerate(l2g)}
    hoff, pins, hw = [0], [], []
    for e in range(a["E"]):
        kept = [loc[v] for v in a["pins"][a["hoff"][e]:a["hoff"][e + 1]] if v in loc]
        if len(kept) < 2:
            continue
        pins += kept
        hoff.append(len(pins))
        hw.append(int(a["hw"][e]))
    nw = [int(a["nw"][v]) for v in l2g]
    return l2g, hoff, pins, nw, hw


def test_subgraph_restated(rng):
    # net splitting (reading C16) against its definition, on random weighted hypergraphs and
    # parts, plus a hyperedge left with exactly one pin in the part (dropped) and one left with
    # two (kept)
    cases = []
    for _ in range(20):
        N = int(rng.integers(5, 60))
        _, hoff, pins, nw, hw = random_hg(rng, N, int(rng.integers(1, 2 * N)), dmax=6,
                                         weights=True, hweights=True)
        part = rng.integers(0, 3, size=N).astype(np.int32)
        cases.append((N, hoff, pins, nw, hw, part))
    # e0 = {0,1,2}: one pin (2) in part 1; e1 = {2,3}: both in part 1; e2 = {0,3,4}: pins 3, 4
    cases.append((5, np.array([0, 3, 5, 8], np.int32), np.array([0, 1, 2, 2, 3, 0, 3, 4], np.int32),
                  np.array([1, 2, 3, 4, 5], np.int32), np.array([7, 8, 9], np.int32),
                  np.array([0, 0, 1, 1, 1], np.int32)))
    for N, hoff, pins, nw, hw, part in cases:
        h = oracle.Hypergraph.from_csr(N, hoff, pins, nw, hw)
        a = h.arrays()
        for j in range(int(part.max()) + 1):
            s, l2g = oracle.subgraph(h, part, j)
            want_l2g, want_hoff, want_pins, want_nw, want_hw = _subgraph_restated(a, part, j)
            b = s.arrays()
            assert l2g.tolist() == want_l2g
            assert b["hoff"].tolist() == want_hoff and b["pins"].tolist() == want_pins
            assert b["nw"].tolist() == want_nw and b["hw"].tolist() == want_hw
    # the constructed case, part 1: nodes 2, 3, 4 -> 0, 1, 2; e0 keeps only node 2 (dropped),
    # e1 -> {0, 1} weight 8, e2 -> {1, 2} weight 9
    h = oracle.Hypergraph.from_csr(*cases[-1][:5])
    s, l2g = oracle.subgraph(h, cases[-1][5], 1)
    b = s.arrays()
    assert l2g.tolist() == [2, 3, 4] and b["hoff"].tolist() == [0, 2, 4]
    assert b["pins"].tolist() == [0, 1, 1, 2] and b["hw"].tolist() == [8, 9]
    assert b["nw"].tolist() == [3, 4, 5]


def test_kway_trivial_and_invalid():
    h = oracle.Hypergraph.from_dict(synth.uniform(100, 100, 2, 4, seed=1))
    part, st = oracle.partition(h, 1)
    assert st == 0 and not part.any()
    part, st = oracle.partition(h, 3)  # any k >= 1 (readings G1-G2)
    assert part.min() >= 0 and part.max() < 3
