"""C ABI checks that need no GPU: the library builds for sm_103a, exports every declared symbol,
and rejects malformed input on the host before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2012_13618_gb300 as bp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "bipart.h")).read()
    return sorted(set(re.findall(r"\b(bipart_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = bp.load()
    names = declared_symbols()
    assert "bipart_create" in names and "bipart_partition" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(bp.SYMBOLS), set(names) - set(bp.SYMBOLS)


def _create_raw(N, hoff, pins, nw=None, hw=None):
    lib = bp.load()
    arr = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.int32)
    hoff, pins, nw, hw = arr(hoff), arr(pins), arr(nw), arr(hw)
    ptr = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)
    out = ctypes.c_void_p()
    rc = lib.bipart_create(N, hoff.size - 1, ptr(hoff), ptr(pins), ptr(nw), ptr(hw), None,
                           ctypes.byref(out))
    return rc, out


@pytest.mark.parametrize("case", [
    dict(N=4, hoff=[1, 2], pins=[0, 1]),                      # offsets[0] != 0
    dict(N=4, hoff=[0, 3, 2], pins=[0, 1, 2]),                # decreasing offsets
    dict(N=4, hoff=[0, 2], pins=[0, 4]),                      # pin out of range
    dict(N=4, hoff=[0, 2], pins=[-1, 2]),                     # negative pin
    dict(N=3, hoff=[0, 2], pins=[0, 1], nw=[1, 0, 1]),        # node weight < 1
    dict(N=3, hoff=[0, 2], pins=[0, 1], hw=[0]),              # hyperedge weight < 1
    dict(N=3, hoff=[0, 2], pins=[0, 1], nw=[2**30, 2**30, 1]),  # node weight sum >= 2^31
])
def test_create_rejects_malformed_csr(case):
    rc, out = _create_raw(case["N"], case["hoff"], case["pins"], case.get("nw"), case.get("hw"))
    assert rc == bp.ERR_INVALID_CSR
    assert not out.value
    assert bp.load().bipart_last_error()


@pytest.mark.parametrize("where", ["pins", "offsets", "nw", "hw"])
def test_large_malformed_csr_reports_first_offender(where):
    # arrays long enough for the validation to run in parallel chunks: the reported index must
    # be the first offending one, as a sequential pass would find it
    N, E = 3_000_000, 1_500_000
    hoff = np.arange(0, 2 * E + 1, 2, dtype=np.int32)
    pins = (np.arange(2 * E, dtype=np.int64) % N).astype(np.int32)
    nw = np.ones(N, np.int32)
    hw = np.ones(E, np.int32)
    first = {"pins": 1_345_678, "offsets": 834_567, "nw": 2_222_222, "hw": 811_111}[where]
    later = first + 600_000  # a later chunk fails too
    if where == "pins":
        pins[first] = N
        pins[later] = -3
    elif where == "offsets":
        hoff[first + 1] = hoff[first] - 1
        hoff[later + 1] = hoff[later] - 1
    elif where == "nw":
        nw[first] = 0
        nw[later] = -1
    else:
        hw[first] = 0
        hw[later] = 0
    rc, out = _create_raw(N, hoff, pins, nw, hw)
    assert rc == bp.ERR_INVALID_CSR and not out.value
    msg = bp.load().bipart_last_error().decode()
    if where in ("pins", "offsets"):
        assert str(first) in msg and str(later) not in msg, msg


def test_null_arguments():
    lib = bp.load()
    hoff = np.array([0, 2], np.int32)
    pins = np.array([0, 1], np.int32)
    rc = lib.bipart_create(2, 1, ctypes.c_void_p(hoff.ctypes.data), ctypes.c_void_p(pins.ctypes.data),
                           None, None, None, None)
    assert rc == bp.ERR_INVALID_ARG
    rc = lib.bipart_create(-1, 1, None, None, None, None, None, ctypes.byref(ctypes.c_void_p()))
    assert rc == bp.ERR_INVALID_ARG
    assert lib.bipart_partition(None, 2, 0.1, 0, 25, 2, None) == bp.ERR_INVALID_ARG
    assert lib.bipart_cut(None, None, None) == bp.ERR_INVALID_ARG
    lib.bipart_destroy(None)


def test_valid_input_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, out = _create_raw(3, [0, 2, 3], [0, 1, 2])
    assert rc == bp.ERR_CUDA and not out.value


def test_batch_and_server_argument_checks():
    lib = bp.load()
    assert lib.bipart_partition_batch(-1, None, None, None, None, 0) == bp.ERR_INVALID_ARG
    assert lib.bipart_partition_batch(2, None, None, None, None, 0) == bp.ERR_INVALID_ARG
    assert lib.bipart_partition_batch(0, None, None, None, None, 0) == bp.OK
    assert lib.bipart_server_create(0, 2, None) == bp.ERR_INVALID_ARG
    assert lib.bipart_server_submit(None, None, None, None, None) == bp.ERR_INVALID_ARG
    assert lib.bipart_server_wait(None, 1, 0, None, None, None) == bp.ERR_INVALID_ARG
    assert lib.bipart_server_stats(None, None, None) == bp.ERR_INVALID_ARG
    lib.bipart_server_destroy(None)
    # tuning: bad sizes are rejected, an empty batch has nothing to tune
    assert lib.bipart_batch_tune(-1, None, None, None) == bp.ERR_INVALID_ARG
    assert lib.bipart_batch_tune(2, None, None, None) == bp.ERR_INVALID_ARG
    chosen = np.full(8, 7, np.int32)
    assert lib.bipart_batch_tune(0, None, None, ctypes.c_void_p(chosen.ctypes.data)) == bp.OK
    assert not chosen.any()
    lib.bipart_batch_release()  # nothing kept yet: a no-op
    # refinement on a kept hierarchy needs a handle
    assert lib.bipart_refine_kept(None, 0.1, 2, None) == bp.ERR_INVALID_ARG


def test_params_validation_before_any_device_work():
    # any k >= 1 is valid (readings G1-G2); k <= 0 and unknown flag bits are rejected on the host
    lib = bp.load()
    g = {"N": 4, "hoff": [0, 2, 4], "pins": [0, 1, 2, 3]}
    for k, flags in [(0, 0), (-3, 0), (2, 4), (3, 1 << 5)]:
        inst, keep = bp._instance(g)
        par = bp.Params(k, 0.1, 0, 25, 2, flags)
        out = np.empty(4, np.int32)
        outs = (ctypes.c_void_p * 1)(out.ctypes.data)
        sts = np.zeros(1, np.int32)
        rc = lib.bipart_partition_batch(1, ctypes.byref(inst), ctypes.byref(par), outs,
                                        ctypes.c_void_p(sts.ctypes.data), 1)
        assert rc == bp.ERR_INVALID_ARG, (k, flags, rc)
    assert lib.bipart_partition_ex(None, None, None) == bp.ERR_INVALID_ARG


def test_batch_prechecks_without_gpu():
    # sizes, pointers, hedge_offsets[0] and hedge_offsets[E] are checked on the host before any
    # device work: an all-invalid batch reports its first instance's error with no GPU present
    lib = bp.load()
    cases = [
        (dict(N=-1, hoff=[0, 2], pins=[0, 1]), bp.ERR_INVALID_ARG),      # negative size
        (dict(N=4, hoff=[1, 2], pins=[0, 1]), bp.ERR_INVALID_CSR),       # offsets[0] != 0
        (dict(N=4, hoff=[0, -2], pins=[0, 1]), bp.ERR_INVALID_CSR),      # offsets[E] < 0
        (dict(N=4, hoff=[0, 2], pins=None), bp.ERR_INVALID_ARG),         # pins NULL with P > 0
    ]
    for case, code in cases:
        g = dict(case)
        keep = [np.ascontiguousarray(g["hoff"], np.int32),
                None if g["pins"] is None else np.ascontiguousarray(g["pins"], np.int32)]
        inst = bp.Instance(g["N"], keep[0].size - 1, ctypes.c_void_p(keep[0].ctypes.data),
                           None if keep[1] is None else ctypes.c_void_p(keep[1].ctypes.data), None, None)
        par = bp.Params(2, 0.1, 0, 25, 2, 0)
        out = np.empty(4, np.int32)
        outs = (ctypes.c_void_p * 1)(out.ctypes.data)
        sts = np.zeros(1, np.int32)
        rc = lib.bipart_partition_batch(1, ctypes.byref(inst), ctypes.byref(par), outs,
                                        ctypes.c_void_p(sts.ctypes.data), 1)
        assert rc == code and sts[0] == code, (case, rc, sts[0])
        assert lib.bipart_last_error().startswith(b"instance 0: ")
