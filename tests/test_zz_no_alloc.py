"""bipart_cut_noalloc: the cut entry point for callers that cannot allocate device memory (for
example an application whose own pool owns all of HBM, or a loop that cannot afford an
allocation's synchronisation).  It must agree exactly with bipart_cut -- the arithmetic is
integer -- on two calls in a row that share its fixed scratch array.  This file is collected last
so a failure here cannot hide the other GPU tests."""
import ctypes

import numpy as np
import pytest

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


def test_cut_noalloc_matches_cut_two_calls(torch_cuda):
    torch = torch_cuda
    import paper_2012_13618_gb300 as bp
    cases = [(synth.c1_netlist(N=60_000), (2, 16)), (synth.rownet(40_000, 40_000, seed=5), (4, 64))]
    for g, ks in cases:
        with bp.create_from(g) as h:
            hoff, pins = _dev(torch, g["hoff"]), _dev(torch, g["pins"])
            hw = None
            for k in ks:
                parts, st = h.partition(k, 0.05, "LDH", 25, 2)
                want = h.cut(parts)
                d_parts = _dev(torch, parts)
                # a second, different partition in the same run: the scratch is reused
                shifted = (parts + 1) % k
                want2 = h.cut(shifted)
                for p_host, exp in ((parts, want), (shifted, want2)):
                    d_parts = _dev(torch, p_host)
                    out = torch.full((1,), -7, dtype=torch.int64, device="cuda")
                    assert bp.cut_noalloc(g["N"], hoff, pins, hw, d_parts, k, out) == 0
                    torch.cuda.synchronize()
                    assert int(out.item()) == exp


def test_cut_noalloc_weighted_and_duplicates(torch_cuda):
    torch = torch_cuda
    import paper_2012_13618_gb300 as bp
    rng = np.random.default_rng(3)
    N, E = 5000, 7000
    deg = rng.integers(0, 40, size=E)
    deg[:5] = 3000  # a few hyperedges handled by whole warps
    hoff = np.zeros(E + 1, np.int32)
    hoff[1:] = np.cumsum(deg)
    pins = rng.integers(0, N, size=int(hoff[-1])).astype(np.int32)
    hw = rng.integers(1, 9, size=E).astype(np.int32)
    parts = rng.integers(0, 8, size=N).astype(np.int32)
    with bp.create(N, hoff, pins, None, hw) as h:
        want = h.cut(parts)
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


def test_cut_noalloc_rejects_sizes_beyond_limit(torch_cuda):
    import paper_2012_13618_gb300 as bp
    lib = bp.load()
    out = ctypes.c_void_p(1)
    assert lib.bipart_cut_noalloc(10, (1 << 22) + 1, out, out, None, out, 2, out, None) == bp.ERR_INVALID_ARG
    assert b"scratch limit" in lib.bipart_last_error()
    assert lib.bipart_cut_noalloc(10, 5, out, out, None, out, 65, out, None) == bp.ERR_INVALID_ARG
