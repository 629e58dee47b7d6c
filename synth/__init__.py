"""Seeded synthetic hypergraph workloads (inputs only; no partitioning arithmetic).

Both the CPU oracle and the CUDA path consume these arrays.  The draws live in ``gen.c``
(xoshiro256** seeded by SplitMix64, one stream per hyperedge); this module compiles it on first
use, allocates the CSR arrays and names the workload shapes:

``c0_uniform``   10,000 nodes / 10,000 hyperedges, degree U{2..6}, unit weights (seed 0).
``c1_netlist``   1M nodes with weights U{1..4}, 1.2M nets: 70% degree 2, a geometric tail to 64,
                 0.1% high-fanout nets U{1000..10000}; pins in a +-max(2000, d) window.
``c2_rownet``    row-net model of a 5M x 5M power-law matrix: Zipf(2.1) row lengths on
                 [2, 100000], 20% of pins in 1% hub columns, unit node weights.
``c3_instance``  one instance of the batched workload: netlist shape, N log-uniform [1k, 200k].

Every generator returns a dict with ``N``, ``E``, ``hoff`` (int32[E+1]), ``pins`` (int32[P]),
``nw`` (int32[N] or None for unit weights) and ``hw`` (None: unit hyperedge weights).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "_synth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into an in-tree shared library (host code only, portable C)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            p32 = ctypes.POINTER(ctypes.c_int32)
            p64 = ctypes.POINTER(ctypes.c_int64)
            pd = ctypes.POINTER(ctypes.c_double)
            lib.synth_uniform_degrees.argtypes = [u64, i32, i32, i32, i32, p32]
            lib.synth_uniform_pins.argtypes = [u64, i32, i32, i32, i32, p64, p32]
            lib.synth_netlist_degrees.argtypes = [u64, i32, i32, dbl, dbl, i32, i32, i32, i32, p32]
            lib.synth_netlist_pins.argtypes = [u64, i32, i32, dbl, dbl, i32, i32, i32, i32, p64, p32]
            lib.synth_node_weights.argtypes = [u64, i32, i32, i32, p32]
            lib.synth_rownet_degrees.argtypes = [u64, i32, i32, dbl, i32, i32, p32]
            lib.synth_rownet_pins.argtypes = [u64, i32, i32, dbl, i32, i32, dbl, dbl, p64, p32]
            lib.synth_uniform01.argtypes = [u64, u64, i32, pd]
            _lib = lib
    return _lib


def _p32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _p64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _csr_from_degrees(deg: np.ndarray):
    off64 = np.zeros(deg.size + 1, dtype=np.int64)
    np.cumsum(deg, out=off64[1:])
    if off64[-1] >= 2**31:
        raise ValueError("workload exceeds int32 pin offsets")
    pins = np.empty(int(off64[-1]), dtype=np.int32)
    return off64, pins


def uniform(N: int, E: int, dmin: int, dmax: int, seed: int) -> dict:
    lib = _load()
    deg = np.empty(E, dtype=np.int32)
    if lib.synth_uniform_degrees(seed, N, E, dmin, dmax, _p32(deg)) != 0:
        raise ValueError("bad uniform parameters")
    off64, pins = _csr_from_degrees(deg)
    if lib.synth_uniform_pins(seed, N, E, dmin, dmax, _p64(off64), _p32(pins)) != 0:
        raise RuntimeError("uniform pin generation failed")
    return dict(N=N, E=E, hoff=off64.astype(np.int32), pins=pins, nw=None, hw=None)


def netlist(N: int, E: int, seed: int, p2=0.70, p_hi=0.001, hi_lo=1000, hi_hi=10000,
            tail_cap=64, win=2000, wmin=1, wmax=4) -> dict:
    lib = _load()
    deg = np.empty(E, dtype=np.int32)
    args = (seed, N, E, p2, p_hi, hi_lo, hi_hi, tail_cap, win)
    if lib.synth_netlist_degrees(*args, _p32(deg)) != 0:
        raise ValueError("bad netlist parameters")
    off64, pins = _csr_from_degrees(deg)
    if lib.synth_netlist_pins(*args, _p64(off64), _p32(pins)) != 0:
        raise RuntimeError("netlist pin generation failed")
    nw = None
    if not (wmin == 1 and wmax == 1):
        nw = np.empty(N, dtype=np.int32)
        lib.synth_node_weights(seed, N, wmin, wmax, _p32(nw))
    return dict(N=N, E=E, hoff=off64.astype(np.int32), pins=pins, nw=nw, hw=None)


def rownet(R: int, C: int, seed: int, alpha=2.1, lmin=2, lmax=100000, p_hub=0.2,
           hub_share=0.01) -> dict:
    lib = _load()
    deg = np.empty(R, dtype=np.int32)
    if lib.synth_rownet_degrees(seed, R, C, alpha, lmin, lmax, _p32(deg)) != 0:
        raise ValueError("bad rownet parameters")
    off64, pins = _csr_from_degrees(deg)
    if lib.synth_rownet_pins(seed, R, C, alpha, lmin, lmax, p_hub, hub_share, _p64(off64),
                             _p32(pins)) != 0:
        raise RuntimeError("rownet pin generation failed")
    return dict(N=C, E=R, hoff=off64.astype(np.int32), pins=pins, nw=None, hw=None)


def uniform01(seed: int, stream: int, n: int) -> np.ndarray:
    lib = _load()
    out = np.empty(n, dtype=np.float64)
    lib.synth_uniform01(seed, stream, n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


# ------------------------------------------------------------------ named workloads
def c0_uniform(seed: int = 0) -> dict:
    """10,000 nodes, 10,000 hyperedges, degree U{2..6}, unit weights."""
    return uniform(10_000, 10_000, 2, 6, seed)


def c1_netlist(seed: int = 1, N: int = 1_000_000) -> dict:
    """Netlist-like: N nodes (weights U{1..4}), 1.2N nets; defaults give the 1M-node case."""
    return netlist(N, int(1.2 * N), seed)


def c2_rownet(seed: int = 2, rows: int = 5_000_000) -> dict:
    """Row-net model of a rows x rows power-law matrix (Zipf 2.1 rows, 20% hub pins)."""
    return rownet(rows, rows, seed)


def c3_size(i: int) -> int:
    """Node count of batched instance i: log-uniform over [1k, 200k]."""
    u = uniform01(3_000_000 + i, 1 << 42, 1)[0]
    return int(round(math.exp(math.log(1_000) + u * (math.log(200_000) - math.log(1_000)))))


def c3_instance(i: int, N: int | None = None) -> dict:
    """Batched instance i: netlist shape with N nodes, E = floor(1.2 N), fanout clipped to N."""
    if N is None:
        N = c3_size(i)
    E = int(1.2 * N)
    hi_lo = min(1000, N // 4)
    hi_hi = min(10000, N // 2)
    return netlist(N, E, 3_000_000 + i, hi_lo=hi_lo, hi_hi=hi_hi, tail_cap=min(64, N))


def num_pins(g: dict) -> int:
    return int(g["hoff"][-1])
