"""Handle creation on the GPU: the copied CSR is checked by a bounded device kernel before any
other kernel reads it, and a failed check falls back to the host pass for the exact error.  Both
entry points (host arrays, device arrays) must give the oracle's bisection on valid input and
INVALID_CSR on malformed input."""

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
    import paper_2012_13618_gb300 as bp
    bp.use_torch_allocator()
    yield


def _bp():
    import paper_2012_13618_gb300 as bp
    return bp


def _dev(a):
    import torch
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def _weighted(seed, N=3000, E=2500):
    rng = np.random.default_rng(seed)
    deg = rng.integers(0, 9, size=E)
    hoff = np.zeros(E + 1, np.int32)
    hoff[1:] = np.cumsum(deg)
    pins = rng.integers(0, N, size=int(hoff[-1])).astype(np.int32)
    nw = rng.integers(1, 7, size=N).astype(np.int32)
    hw = rng.integers(1, 5, size=E).astype(np.int32)
    return dict(N=N, E=E, hoff=hoff, pins=pins, nw=nw, hw=hw)


@pytest.mark.parametrize("seed", [1, 2])
def test_host_and_device_arrays_match_oracle(seed):
    bp = _bp()
    g = _weighted(seed)
    ref = oracle.bisect(oracle.Hypergraph.from_dict(g), 0.1, "LDH", 25, 2)
    want = ref["side"].astype(np.int32)
    with bp.create(g["N"], g["hoff"], g["pins"], g["nw"], g["hw"]) as h:
        parts, st = h.partition(2, 0.1, "LDH", 25, 2)
        assert np.array_equal(parts, want) and st == ref["status"]
    with bp.create_device(g["N"], _dev(g["hoff"]), _dev(g["pins"]), _dev(g["nw"]), _dev(g["hw"])) as h:
        parts, st = h.partition(2, 0.1, "LDH", 25, 2)
        assert np.array_equal(parts, want) and st == ref["status"]


def test_device_arrays_without_hyperedges():
    bp = _bp()
    with bp.create_device(5, _dev(np.zeros(1, np.int32)), _dev(np.zeros(1, np.int32))) as h:
        parts, st = h.partition(2)
        assert st == 0 and parts.size == 5


# every case keeps hoff[E] <= len(pins), the documented length of the pin array
MALFORMED = [
    dict(N=4, hoff=[0, 3, 2], pins=[0, 1, 2]),                  # decreasing offsets
    dict(N=4, hoff=[0, 2], pins=[0, 4]),                        # pin out of range
    dict(N=4, hoff=[0, 2], pins=[-1, 2]),                       # negative pin
    dict(N=3, hoff=[0, 2], pins=[0, 1], nw=[1, 0, 1]),          # node weight < 1
    dict(N=3, hoff=[0, 2], pins=[0, 1], hw=[0]),                # hyperedge weight < 1
    dict(N=3, hoff=[0, 2], pins=[0, 1], nw=[2**30, 2**30, 1]),  # node weight sum >= 2^31
]


@pytest.mark.parametrize("case", MALFORMED)
def test_malformed_host_arrays_rejected(case):
    bp = _bp()
    with pytest.raises(bp.BipartError) as ei:
        bp.create(case["N"], case["hoff"], case["pins"], case.get("nw"), case.get("hw"))
    assert ei.value.code == bp.ERR_INVALID_CSR


@pytest.mark.parametrize("case", MALFORMED)
def test_malformed_device_arrays_rejected(case):
    bp = _bp()
    with pytest.raises(bp.BipartError) as ei:
        bp.create_device(case["N"], _dev(case["hoff"]), _dev(case["pins"]), _dev(case.get("nw")),
                         _dev(case.get("hw")))
    assert ei.value.code == bp.ERR_INVALID_CSR


@pytest.mark.parametrize("where", ["pins", "offsets"])
def test_malformed_large_host_arrays_name_first_offender(where):
    # the device check fails, the host pass then names the first offending index
    bp = _bp()
    N, E = 3_000_000, 1_500_000
    hoff = np.arange(0, 2 * E + 1, 2, dtype=np.int32)
    pins = (np.arange(2 * E, dtype=np.int64) % N).astype(np.int32)
    first = {"pins": 1_345_678, "offsets": 834_567}[where]
    later = first + 600_000
    if where == "pins":
        pins[first] = N
        pins[later] = -3
    else:
        hoff[first + 1] = hoff[first] - 1
        hoff[later + 1] = hoff[later] - 1
    with pytest.raises(bp.BipartError) as ei:
        bp.create(N, hoff, pins)
    assert ei.value.code == bp.ERR_INVALID_CSR
    msg = str(ei.value)
    assert str(first) in msg and str(later) not in msg, msg


def test_valid_after_malformed_on_same_stream():
    # a rejected creation leaves nothing behind that changes the next one
    bp = _bp()
    with pytest.raises(bp.BipartError):
        bp.create(4, [0, 2], [0, 4])
    g = synth.uniform(2000, 1500, 2, 6, seed=9)
    ref = oracle.bisect(oracle.Hypergraph.from_dict(g), 0.1, "LDH", 25, 2)
    with bp.create_from(g) as h:
        parts, st = h.partition(2, 0.1, "LDH", 25, 2)
        assert np.array_equal(parts, ref["side"].astype(np.int32))


def _batch_raw(graphs, params, workers=2):
    import ctypes
    bp = _bp()
    n, keep, insts, pars = bp._batch_args(graphs, params)
    outs = [np.full(max(int(g["N"]), 1), -7, np.int32) for g in graphs]
    out_ptrs = (ctypes.c_void_p * n)(*[o.ctypes.data for o in outs])
    st = np.zeros(n, np.int32)
    rc = bp.load().bipart_partition_batch(n, ctypes.cast(insts, ctypes.c_void_p), ctypes.cast(pars, ctypes.c_void_p),
                                          ctypes.cast(out_ptrs, ctypes.c_void_p),
                                          ctypes.c_void_p(st.ctypes.data), workers)
    return rc, [o[: int(g["N"])] for o, g in zip(outs, graphs)], st, bp.load().bipart_last_error().decode()


def _malformed_like(g, what):
    # a copy of g with one defect, keeping hoff[E] == len(pins)
    g = {k: (None if v is None else (np.array(v, copy=True) if isinstance(v, np.ndarray) else v))
         for k, v in g.items()}
    if what == "pin":
        g["pins"][len(g["pins"]) // 2] = g["N"] + 5
    elif what == "offsets":
        e = g["E"] // 2
        g["hoff"][e + 1] = g["hoff"][e] - 1
    elif what == "nw":
        g["nw"] = np.ones(g["N"], np.int32)
        g["nw"][g["N"] // 3] = 0
    return g


def test_batch_malformed_instances_reported_others_exact():
    # malformed instances among valid ones on the persistent block path: each malformed one gets
    # INVALID_CSR and keeps its output untouched, every valid one equals the oracle
    bp = _bp()
    base = [synth.uniform(1500 + 100 * i, 1400 + 90 * i, 2, 6, seed=40 + i) for i in range(6)]
    kinds = [None, "pin", None, "offsets", "nw", None]
    graphs = [g if k is None else _malformed_like(g, k) for g, k in zip(base, kinds)]
    p = dict(k=2, eps=0.05, policy="LDH", levels=25, iters=2)
    rc, parts, st, msg = _batch_raw(graphs, p)
    assert rc == bp.ERR_INVALID_CSR and "instance 1" in msg, msg
    for i, (g, k) in enumerate(zip(graphs, kinds)):
        if k is None:
            ref = oracle.bisect(oracle.Hypergraph.from_dict(g), 0.05, "LDH", 25, 2)
            assert np.array_equal(parts[i], ref["side"].astype(np.int32)) and st[i] == ref["status"], i
        else:
            assert st[i] == bp.ERR_INVALID_CSR and (parts[i] == -7).all(), (i, k)


def test_server_rejects_bad_requests_without_touching_others():
    # a request with bad parameters completes at once; malformed CSRs complete with INVALID_CSR,
    # whether they ran in a micro-batch or alone; the valid requests equal the oracle
    bp = _bp()
    base = [synth.uniform(1200 + 50 * i, 1100 + 40 * i, 2, 6, seed=70 + i) for i in range(16)]
    kinds = [None] * 16
    kinds[3], kinds[8], kinds[12] = "pin", "offsets", "nw"
    graphs = [g if k is None else _malformed_like(g, k) for g, k in zip(base, kinds)]
    with bp.Server(hbm_budget_bytes=0, workers=1) as srv:
        tickets = [srv.submit(g, k=2, eps=0.05) for g in graphs]
        bad_k = srv.submit(base[0], k=0, eps=0.05)
        for i, t in enumerate(tickets):
            parts, st, _, _ = srv.wait(t)
            if kinds[i] is None:
                ref = oracle.bisect(oracle.Hypergraph.from_dict(graphs[i]), 0.05, "LDH", 25, 2)
                assert np.array_equal(parts, ref["side"].astype(np.int32)) and st == ref["status"], i
            else:
                assert st == bp.ERR_INVALID_CSR, (i, kinds[i], st)
        _, st, _, _ = srv.wait(bad_k)
        assert st == bp.ERR_INVALID_ARG


def test_batch_staging_mixed_inputs_match_oracle():
    # staged batch inputs: instances with and without weights, no hyperedges, pin arrays that
    # start off a 16-byte boundary; the replayed graph takes new source arrays
    bp = _bp()
    graphs = []
    for i in range(8):
        g = _weighted(100 + i, N=1500 + 200 * i, E=1300 + 150 * i)
        if i % 2:
            g["nw"] = g["hw"] = None
        if i % 3 == 1:
            # a view one element into a larger array: the source is not 16-byte aligned
            buf = np.empty(g["pins"].size + 1, np.int32)
            buf[1:] = g["pins"]
            g["pins"] = buf[1:]
        graphs.append(g)
    graphs.append(dict(N=40, E=0, hoff=np.zeros(1, np.int32), pins=np.zeros(0, np.int32), nw=None, hw=None))
    p = dict(k=2, eps=0.05, policy="LDH", levels=25, iters=2)
    for rep in range(2):  # capture, then replay on copies (new source arrays)
        if rep:
            graphs = [{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in g.items()} for g in graphs]
        parts, st = bp.partition_batch(graphs, p, workers=2)
        for i, g in enumerate(graphs):
            ref = oracle.bisect(oracle.Hypergraph.from_dict(g), 0.05, "LDH", 25, 2)
            assert np.array_equal(parts[i], ref["side"].astype(np.int32)) and st[i] == ref["status"], i
