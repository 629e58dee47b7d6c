"""bipart_cut_noalloc: the cut entry point for callers that cannot allocate device memory (for
example an application whose own pool owns all of HBM, or a loop that cannot afford an
allocation's synchronisation).  Its result must equal the oracle's cut (Sec. 1.1, the arithmetic
is integer) on calls in a row that share its fixed scratch array, on the default stream and on
streams the caller owns.  This file is collected last so a failure here cannot hide the other GPU
tests."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return torch


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def _oracle_cut(N, hoff, pins, hw, parts):
    return oracle.cut(oracle.Hypergraph.from_csr(N, hoff, pins, None, hw), parts)


def test_cut_noalloc_matches_oracle_two_calls(torch_cuda):
    torch = torch_cuda
    import paper_2012_13618_gb300 as bp
    cases = [(synth.c1_netlist(N=60_000), (2, 16)), (synth.rownet(40_000, 40_000, seed=5), (4, 64))]
    for g, ks in cases:
        with bp.create_from(g) as h:
            hoff, pins = _dev(torch, g["hoff"]), _dev(torch, g["pins"])
            for k in ks:
                parts, st = h.partition(k, 0.05, "LDH", 25, 2)
                # a second, different partition in the same run: the scratch is reused
                shifted = (parts + 1) % k
                for p_host in (parts, shifted):
                    exp = _oracle_cut(g["N"], g["hoff"], g["pins"], None, p_host)
                    d_parts = _dev(torch, p_host)
                    out = torch.full((1,), -7, dtype=torch.int64, device="cuda")
                    assert bp.cut_noalloc(g["N"], hoff, pins, None, d_parts, k, out) == 0
                    torch.cuda.synchronize()
                    assert int(out.item()) == exp


def _weighted_case(seed=3):
    rng = np.random.default_rng(seed)
    N, E = 5000, 7000
    deg = rng.integers(0, 40, size=E)
    deg[:5] = 3000  # a few hyperedges handled by whole warps
    hoff = np.zeros(E + 1, np.int32)
    hoff[1:] = np.cumsum(deg)
    pins = rng.integers(0, N, size=int(hoff[-1])).astype(np.int32)
    hw = rng.integers(1, 9, size=E).astype(np.int32)
    parts = rng.integers(0, 8, size=N).astype(np.int32)
    return N, hoff, pins, hw, parts


def test_cut_noalloc_weighted_and_duplicates(torch_cuda):
    torch = torch_cuda
    import paper_2012_13618_gb300 as bp
    N, hoff, pins, hw, parts = _weighted_case()
    want = _oracle_cut(N, hoff, pins, hw, parts)
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(2):
        assert bp.cut_noalloc(N, _dev(torch, hoff), _dev(torch, pins), _dev(torch, hw),
                              _dev(torch, parts), 8, out) == 0
        torch.cuda.synchronize()
        assert int(out.item()) == want
    bad = parts.copy()
    bad[0] = 8
    assert bp.cut_noalloc(N, _dev(torch, hoff), _dev(torch, pins), _dev(torch, hw),
                          _dev(torch, bad), 8, out) == 0
    torch.cuda.synchronize()
    assert int(out.item()) == -1
    # a hyperedge weight below 1 is rejected the same way (bipart_create refuses it too)
    for w in (-3, 0):
        bad_hw = hw.copy()
        bad_hw[17] = w
        assert bp.cut_noalloc(N, _dev(torch, hoff), _dev(torch, pins), _dev(torch, bad_hw),
                              _dev(torch, parts), 8, out) == 0
        torch.cuda.synchronize()
        assert int(out.item()) == -1
    # and the next valid call is not affected by the flag the rejected one raised
    assert bp.cut_noalloc(N, _dev(torch, hoff), _dev(torch, pins), _dev(torch, hw),
                          _dev(torch, parts), 8, out) == 0
    torch.cuda.synchronize()
    assert int(out.item()) == want


def test_cut_noalloc_on_caller_streams(torch_cuda):
    # two calls in a row on a non-blocking stream the caller owns, then one on a second stream
    # ordered after the first: ordered calls share the scratch safely
    torch = torch_cuda
    import paper_2012_13618_gb300 as bp
    N, hoff, pins, hw, parts = _weighted_case(seed=8)
    other = (parts * 5 + 3) % 8
    third = (parts + 2) % 6
    d_hoff, d_pins, d_hw = _dev(torch, hoff), _dev(torch, pins), _dev(torch, hw)
    d_parts, d_other, d_third = _dev(torch, parts), _dev(torch, other), _dev(torch, third)
    outs = torch.full((3,), -7, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with torch.cuda.stream(s1):
        assert bp.cut_noalloc(N, d_hoff, d_pins, d_hw, d_parts, 8, outs[0:1], stream=s1) == 0
        assert bp.cut_noalloc(N, d_hoff, d_pins, d_hw, d_other, 8, outs[1:2], stream=s1) == 0
    s2.wait_stream(s1)
    with torch.cuda.stream(s2):
        assert bp.cut_noalloc(N, d_hoff, d_pins, d_hw, d_third, 6, outs[2:3], stream=s2) == 0
    torch.cuda.synchronize()
    want = [_oracle_cut(N, hoff, pins, hw, p) for p in (parts, other, third)]
    assert outs.cpu().tolist() == want


def test_cut_noalloc_rejects_sizes_beyond_limit(torch_cuda):
    import paper_2012_13618_gb300 as bp
    lib = bp.load()
    out = ctypes.c_void_p(1)
    assert lib.bipart_cut_noalloc(10, (1 << 22) + 1, out, out, None, out, 2, out, None) == bp.ERR_INVALID_ARG
    assert b"scratch limit" in lib.bipart_last_error()
    assert lib.bipart_cut_noalloc(10, 5, out, out, None, out, 65, out, None) == bp.ERR_INVALID_ARG
