"""Design-space sweep (Sec. 4.3): one hypergraph partitioned under every combination of
coarsening levels, refinement iterations and matching policy, and the Pareto frontier of
(run time, cut).  Because every configuration is deterministic, the frontier is reproducible.

The hypergraph is uploaded once.  Coarsening depends only on (levels, policy), so the partitions
of one (levels, policy) group share one hierarchy: its first configuration partitions in full and
the others re-run only Algorithm 3 and the refinement on the kept levels (bipart_refine_kept),
which gives the same partitions.  Each configuration's run time is then measured alone on the
resident handle as a full bisection (warm: the launch plan of that configuration is captured
first).
"""
from __future__ import annotations

import itertools
import time

from . import create_from


def pareto(points):
    """Indices of the points (time, cut) not dominated by another point (lower or equal in both,
    lower in one)."""
    idx = []
    for i, (ti, ci) in enumerate(points):
        dominated = any((tj <= ti and cj <= ci) and (tj < ti or cj < ci)
                        for j, (tj, cj) in enumerate(points) if j != i)
        if not dominated:
            idx.append(i)
    return idx


def sweep(g, levels=(5, 10, 25), iters=(0, 1, 2, 4), policies=("LDH", "HDH", "RAND"), eps=0.1,
          k=2, time_each=True, repeats=3, workers=0):
    """Returns (results, frontier): results = list of dicts (levels, iters, policy, cut, status,
    ms), frontier = indices of the Pareto-optimal results."""
    if k != 2:
        raise ValueError("the sweep runs bisections (k = 2)")
    configs = [dict(k=k, eps=eps, policy=p, levels=l, iters=i)
               for p, l, i in itertools.product(policies, levels, iters)]
    results = []
    with create_from(g) as h:
        # partitions: one coarsening per (levels, policy) group, the other iteration counts on
        # the kept hierarchy
        parts, st = [], []
        for pol, lev in itertools.product(policies, levels):
            group = [c for c in configs if c["policy"] == pol and c["levels"] == lev]
            for j, c in enumerate(group):
                if j == 0:
                    pp, ss = h.partition(k, eps, pol, lev, c["iters"])
                else:
                    pp, ss = h.refine_kept(eps, c["iters"])
                parts.append(pp)
                st.append(ss)
        for c, p, s in zip(configs, parts, st):
            r = dict(levels=c["levels"], iters=c["iters"], policy=c["policy"], cut=h.cut(p),
                     status=int(s), parts=p, ms=None)
            if time_each:
                h.partition(k, eps, c["policy"], c["levels"], c["iters"])  # eager, records sizes
                h.partition(k, eps, c["policy"], c["levels"], c["iters"])  # captures the plan
                best = None
                for _ in range(repeats):
                    t0 = time.perf_counter()
                    h.partition(k, eps, c["policy"], c["levels"], c["iters"])
                    dt = 1000 * (time.perf_counter() - t0)
                    best = dt if best is None else min(best, dt)
                r["ms"] = best
            results.append(r)
    front = pareto([(r["ms"] if r["ms"] is not None else 0.0, r["cut"]) for r in results])
    return results, front
