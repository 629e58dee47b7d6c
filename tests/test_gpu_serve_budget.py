"""Serving under an HBM budget: the admission estimate of a request against the device memory its
workspace really allocates (counted through the allocator hooks), and the server's live device
memory against the budget while a trace that needs queueing runs.  Every result is also checked
against the oracle."""
import threading

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def estimate_bytes(g):
    # the server's admission estimate of a request (64 P + 96 E + 96 N + 8 MiB)
    return 64 * int(g["hoff"][-1]) + 96 * (int(g["E"]) + int(g["N"])) + (8 << 20)


class Counting:
    """Allocator hooks over PyTorch's caching allocator that keep the live and peak bytes."""

    def __init__(self, bp):
        import torch
        self.torch = torch
        self.lock = threading.Lock()
        self.sizes = {}
        self.live = 0
        self.peak = 0
        self._a = bp._ALLOC(self._alloc)
        self._f = bp._FREE(self._free)

    def _alloc(self, ctx, nbytes, stream):
        try:
            p = int(self.torch.cuda.caching_allocator_alloc(int(nbytes), 0, int(stream or 0)))
        except Exception:
            return None
        with self.lock:
            self.sizes[p] = int(nbytes)
            self.live += int(nbytes)
            self.peak = max(self.peak, self.live)
        return p

    def _free(self, ctx, ptr, nbytes, stream):
        with self.lock:
            self.live -= self.sizes.pop(int(ptr), 0)
        self.torch.cuda.caching_allocator_delete(int(ptr))

    def reset_peak(self):
        with self.lock:
            self.peak = self.live


@pytest.fixture()
def counting():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2012_13618_gb300 as bp
    c = Counting(bp)
    bp._check(bp.load().bipart_set_allocator(c._a, c._f, None))
    yield c
    bp.use_default_allocator()


def requests():
    out = []
    for i, (kind, n) in enumerate([("net", 2_000), ("net", 20_000), ("net", 150_000), ("row", 3_000),
                                   ("row", 40_000), ("row", 120_000)]):
        g = synth.c3_instance(7_000 + i, N=n) if kind == "net" else synth.rownet(n, n, seed=7_000 + i)
        for k in (2, 4, 16):
            out.append((g, k))
    return out


def test_estimate_bounds_what_a_request_allocates(counting):
    # one worker under a (large) budget: each request runs alone on a workspace that is emptied
    # after it, so the peak over a request is what that request allocated
    import paper_2012_13618_gb300 as bp
    with bp.Server(hbm_budget_bytes=1 << 40, workers=1) as srv:
        for g, k in requests():
            srv.wait(srv.submit(g, k=2, eps=0.05))  # the worker's workspace exists
            counting.reset_peak()
            base = counting.live
            parts, st, _, _ = srv.wait(srv.submit(g, k=k, eps=0.05))
            assert st >= 0
            used = counting.peak - base
            assert used <= estimate_bytes(g), (g["N"], k, used, estimate_bytes(g))


def test_server_live_memory_stays_within_budget(counting):
    import paper_2012_13618_gb300 as bp
    reqs = requests()
    budget = 2 * max(estimate_bytes(g) for g, _ in reqs)
    refs = [oracle.partition(oracle.Hypergraph.from_dict(g), k, 0.05, "LDH", 25, 2) for g, k in reqs]
    counting.reset_peak()
    base = counting.live
    with bp.Server(hbm_budget_bytes=budget, workers=4) as srv:
        tickets = [srv.submit(g, k=k, eps=0.05) for g, k in reqs]
        for (g, k), t, (ref, rst) in zip(reqs, tickets, refs):
            parts, st, _, _ = srv.wait(t)
            assert np.array_equal(parts, ref) and st == rst
    assert counting.peak - base <= budget, (counting.peak - base, budget)
