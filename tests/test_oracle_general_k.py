"""Pins of the oracle's k-way extension to any k (readings G1-G3; the paper's Algorithm 6 covers
powers of two and is silent on other k and on the per-bisection imbalance).

G1  a subgraph owning the parts [lo, lo + m) puts ceil(m / 2) of them on side 0
G2  targets and limits in proportion: side s may hold max(ceil(W ms / m), floor(W ms (1 + e) / m));
    Algorithm 3 grows P0 while m W0 < m0 W
G3  adaptive imbalance: the largest e' (millionths) with (1 + e')^L <= 1 + e, L = ceil(log2 k)

Checked against exact big-integer / rational arithmetic written here, closed forms for unit
weights, and the structure of the recursion."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _L(k):
    return max(0, (k - 1).bit_length())


@pytest.mark.parametrize("e6", [0, 1, 999, 50_000, 100_000, 999_999, 1_000_000_000])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 8, 9, 64, 1000, (1 << 20) + 1])
def test_adaptive_e6_is_the_largest_fitting_integer(e6, k):
    x = oracle.adaptive_e6(e6, k)
    L = _L(k)
    if L <= 1:
        assert x == e6
        return
    rhs = (10**6 + e6) * 10 ** (6 * (L - 1))
    assert 0 <= x <= e6
    assert (10**6 + x) ** L <= rhs
    assert x == e6 or (10**6 + x + 1) ** L > rhs
    # and it is floor(10^6 ((1 + e)^(1/L) - 1)) up to floating-point error
    approx = 1e6 * ((1 + e6 / 1e6) ** (1.0 / L) - 1)
    assert abs(x - approx) < 1.0 + 1e-9 * approx


def test_adaptive_e6_monotone_in_k():
    prev = None
    for k in range(2, 300):
        x = oracle.adaptive_e6(100_000, k)
        if prev is not None:
            assert x <= prev
        prev = x


def test_limit_part_properties():
    rng = np.random.default_rng(5)
    for _ in range(2000):
        W = int(rng.integers(0, 2**31))
        m = int(rng.integers(2, 2**20))
        ms = int(rng.integers(1, m))
        e6 = int(rng.choice([0, 1, 50_000, 100_000, int(rng.integers(0, 10**9))]))
        lim = oracle.limit_part(W, ms, m, e6)
        share = Fraction(W * ms, m)
        allowed = share * Fraction(10**6 + e6, 10**6)
        assert lim >= share                      # a side can always hold its share
        assert lim <= max(math.ceil(share), allowed)  # and never more than the allowance
        assert lim + 1 > allowed or lim == math.ceil(share)  # the allowance is used in full
        lim1 = oracle.limit_part(W, m - ms, m, e6)
        assert lim + lim1 >= W                   # the two sides can hold everything


def test_limit_part_reduces_to_the_bisection_limit():
    rng = np.random.default_rng(6)
    for _ in range(500):
        W = int(rng.integers(0, 2**31))
        eps = float(rng.choice([0.0, 0.05, 0.1, 0.3, 1.0]))
        e6 = int(math.floor(eps * 1e6 + 0.5))
        assert oracle.limit_part(W, 1, 2, e6) == oracle.limit(W, eps)
        m = 2 * int(rng.integers(1, 1000))
        assert oracle.limit_part(W, m // 2, m, e6) == oracle.limit(W, eps)


@pytest.mark.parametrize("m0,m", [(1, 2), (1, 3), (2, 3), (3, 5), (1, 7), (4, 7)])
def test_initial_target_unit_weights_closed_form(m0, m):
    # unit weights: every round moves exactly s = ceil(sqrt(n)) nodes while P1 has them, so the
    # loop ends after the first round r with m * min(r s, N) >= m0 * N
    g = synth.uniform(900, 1100, 2, 5, seed=31)
    h = oracle.Hypergraph.from_dict(g)
    n = h.N
    s = oracle.ceil_sqrt(n)
    side, rounds = oracle.initial(h, m0, m)
    r = 0
    while m * min(r * s, n) < m0 * n:
        r += 1
    assert rounds == r
    assert int((side == 0).sum()) == min(r * s, n)
    if (m0, m) == (1, 2):
        side2, rounds2 = oracle.initial(h)
        assert rounds2 == rounds and np.array_equal(side2, side)


def test_rebalance_with_two_limits(rng):
    for trial in range(40):
        g = synth.uniform(300, 350, 2, 5, seed=100 + trial)
        g["nw"] = rng.integers(1, 5, size=g["N"]).astype(np.int32)
        h = oracle.Hypergraph.from_dict(g)
        W = int(np.asarray(g["nw"]).sum())
        side = rng.integers(0, 2, size=h.N).astype(np.uint8)
        m = int(rng.integers(3, 9))
        m0 = int(rng.integers(1, m))
        l0 = oracle.limit_part(W, m0, m, 50_000)
        l1 = oracle.limit_part(W, m - m0, m, 50_000)
        st, _ = oracle.rebalance(h, side, l0, l1)
        w0 = int(np.asarray(g["nw"])[side == 0].sum())
        if st == 0:
            assert w0 <= l0 and W - w0 <= l1
        # equal limits: the two-limit form is the single-limit one
        side_a = rng.integers(0, 2, size=h.N).astype(np.uint8)
        side_b = side_a.copy()
        lim = oracle.limit(W, 0.05)
        assert oracle.rebalance(h, side_a, lim) == oracle.rebalance(h, side_b, lim, lim)
        assert np.array_equal(side_a, side_b)


def _check_recursion(h, part, k, e6, policy, levels, iters, lo=0, m=None, nodes=None, W=None):
    """Walks the recursion of G1: the nodes of range [lo, lo + m) are the subgraph; its side 0 is
    exactly the nodes whose final part is below lo + ceil(m / 2), and that side equals the
    stand-alone bisection of the subgraph with target (ceil(m / 2), m).  Returns the sum of the
    bisection cuts of the subtree."""
    if m is None:
        m = k
    if m < 2:
        return 0
    m0 = (m + 1) // 2
    in_range = ((part >= lo) & (part < lo + m)).astype(np.int32)
    s, l2g = oracle.subgraph(h, in_range, 1)
    side = (part[l2g] >= lo + m0).astype(np.uint8)
    r = oracle.bisect(s, policy=policy, levels=levels, iters=iters, keep_levels=False,
                      target=(m0, m), e6=e6)
    assert np.array_equal(r["side"], side)
    total = oracle.cut_bisection(s, side)
    total += _check_recursion(h, part, k, e6, policy, levels, iters, lo, m0)
    total += _check_recursion(h, part, k, e6, policy, levels, iters, lo + m0, m - m0)
    return total


@pytest.mark.parametrize("k", [3, 5, 6, 7, 12])
def test_general_k_recursion_and_cut_identity(k):
    h = oracle.Hypergraph.from_dict(synth.uniform(1500, 1600, 2, 6, seed=21))
    part, st = oracle.partition(h, k, 0.1, "LDH", 25, 2)
    assert part.min() >= 0 and part.max() < k
    assert len(np.unique(part)) == k
    total = _check_recursion(h, part, k, 100_000, 0, 25, 2)
    # reading C17: the lambda-1 cut is the sum of the bisection cuts over the recursion tree
    assert total == oracle.cut(h, part)


def test_power_of_two_k_keeps_the_paper_numbering():
    h = oracle.Hypergraph.from_dict(synth.uniform(1200, 1300, 2, 5, seed=13))
    part, _ = oracle.partition(h, 8, 0.1, "RAND", 25, 2)
    _check_recursion(h, part, 8, 100_000, 4, 25, 2)
    # tree level t splits halves, so the parts of level t are part >> (3 - t)
    r = oracle.bisect(h, 0.1, "RAND", 25, 2, keep_levels=False)
    assert np.array_equal(part >> 2, r["side"].astype(np.int32))


@pytest.mark.parametrize("k", [3, 6, 10])
def test_adaptive_imbalance_bounds_every_part(k):
    # with every bisection held to (1 + e')-times its share, e' of reading G3, a final part weighs
    # at most W (1 + e) / k plus one unit of rounding per tree level
    g = synth.uniform(2000, 2200, 2, 6, seed=41)
    g["nw"] = np.random.default_rng(3).integers(1, 4, size=g["N"]).astype(np.int32)
    h = oracle.Hypergraph.from_dict(g)
    W = int(np.asarray(g["nw"]).sum())
    part, st = oracle.partition(h, k, 0.1, "LDH", 25, 2, adaptive=True)
    if st != 0:
        pytest.skip("a rebalance ran out of candidates")
    wp = np.bincount(part, weights=np.asarray(g["nw"]), minlength=k)
    bound = Fraction(W * 11, 10 * k) + _L(k)
    assert all(Fraction(int(x)) <= bound for x in wp)
    e6 = oracle.adaptive_e6(100_000, k)
    _check_recursion(h, part, k, e6, 0, 25, 2)


def test_kway_k_must_be_positive():
    h = oracle.Hypergraph.from_dict(synth.uniform(100, 100, 2, 4, seed=1))
    for k in (0, -1):
        _, st = oracle.partition(h, k)
        assert st == oracle.ERR_INVALID_ARG
