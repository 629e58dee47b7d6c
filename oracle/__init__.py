"""CPU oracle of BiPart's deterministic multilevel bisection -- TEST INFRASTRUCTURE ONLY.

The arithmetic lives in ``bipart_oracle.c`` (plain sequential C, one function per algorithm of
the paper); this module compiles it and marshals numpy arrays through ctypes.  Only the tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may use it.  It shares no code
with the CUDA path under ``paper_2012_13618_gb300``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bipart_oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

POLICIES = {"LDH": 0, "HDH": 1, "LWD": 2, "HWD": 3, "RAND": 4}
OK, WARN_IMBALANCED, ERR_INVALID_ARG = 0, 1, -1


def build(force: bool = False) -> str:
    """Compile the oracle into an in-tree shared library (portable C11, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC,
                               "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u32 = ctypes.c_uint32
_dbl = ctypes.c_double


def _load():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            sig = {
                "orc_hg_normalise": (_vp, [_i32, _i32, _vp, _vp, _vp, _vp]),
                "orc_hg_free": (None, [_vp]),
                "orc_hg_N": (_i32, [_vp]),
                "orc_hg_E": (_i32, [_vp]),
                "orc_hg_P": (_i32, [_vp]),
                "orc_hg_copy": (None, [_vp, _vp, _vp, _vp, _vp]),
                "orc_hash": (_u32, [_u32]),
                "orc_priority": (_u32, [_vp, _i32, ctypes.c_int]),
                "orc_match": (None, [_vp, ctypes.c_int, _vp]),
                "orc_coarsen": (_vp, [_vp, ctypes.c_int, _vp, _vp]),
                "orc_gains": (None, [_vp, _vp, _vp]),
                "orc_ceil_sqrt": (_i64, [_i64]),
                "orc_initial": (_i32, [_vp, _vp]),
                "orc_refine_iter": (_i32, [_vp, _vp]),
                "orc_limit": (_i64, [_i64, _dbl]),
                "orc_rebalance": (ctypes.c_int, [_vp, _vp, _i64, _vp]),
                "orc_bisect": (_vp, [_vp, _dbl, ctypes.c_int, _i32, _i32]),
                "orc_run_nlev": (_i32, [_vp]),
                "orc_run_level": (_vp, [_vp, _i32]),
                "orc_run_cmap": (None, [_vp, _i32, _vp]),
                "orc_run_match": (None, [_vp, _i32, _vp]),
                "orc_run_side": (None, [_vp, _vp]),
                "orc_run_status": (ctypes.c_int, [_vp]),
                "orc_run_init_rounds": (_i32, [_vp]),
                "orc_run_limit": (_i64, [_vp]),
                "orc_run_free": (None, [_vp]),
                "orc_cut": (_i64, [_vp, _vp]),
                "orc_cut_bisection": (_i64, [_vp, _vp]),
                "orc_subgraph": (_vp, [_vp, _vp, _i32, _vp]),
                "orc_partition": (ctypes.c_int, [_vp, _i32, _dbl, ctypes.c_int, _i32, _i32, _vp]),
                "orc_partition_ex": (ctypes.c_int, [_vp, _i32, _i64, ctypes.c_int, ctypes.c_int,
                                                    _i32, _i32, _vp]),
                "orc_initial_target": (_i32, [_vp, _vp, _i32, _i32]),
                "orc_rebalance2": (ctypes.c_int, [_vp, _vp, _i64, _i64, _vp]),
                "orc_limit_part": (_i64, [_i64, _i32, _i32, _i64]),
                "orc_adaptive_e6": (_i64, [_i64, _i32]),
                "orc_bisect_target": (_vp, [_vp, _i64, _i32, _i32, ctypes.c_int, _i32, _i32]),
                "orc_bisect_ex": (_vp, [_vp, _i64, _i32, _i32, ctypes.c_int, ctypes.c_int, _i32, _i32]),
                "orc_coarsen_ex": (_vp, [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp]),
                "orc_merge_parallel": (None, [_vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _i32arr(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def _e6(eps: float) -> int:
    """eps in millionths, rounded half away from zero like C's llround (eps >= 0)."""
    return int(math.floor(float(eps) * 1e6 + 0.5))


def _policy(p) -> int:
    return POLICIES[p] if isinstance(p, str) else int(p)


class Hypergraph:
    """A normalised hypergraph owned by the oracle (sorted unique pins, >= 2 pins per edge)."""

    def __init__(self, handle, owned=True):
        self._h = handle
        self._owned = owned

    @classmethod
    def from_csr(cls, N, hoff, pins, nw=None, hw=None):
        L = _load()
        hoff = _i32arr(hoff)
        pins = _i32arr(pins)
        nw = _i32arr(nw)
        hw = _i32arr(hw)
        h = L.orc_hg_normalise(int(N), int(hoff.size - 1), _ptr(hoff), _ptr(pins), _ptr(nw),
                               _ptr(hw))
        return cls(h)

    @classmethod
    def from_dict(cls, g):
        return cls.from_csr(g["N"], g["hoff"], g["pins"], g.get("nw"), g.get("hw"))

    def __del__(self):
        if getattr(self, "_owned", False) and self._h and _lib is not None:
            _lib.orc_hg_free(self._h)
            self._h = None

    @property
    def N(self):
        return _load().orc_hg_N(self._h)

    @property
    def E(self):
        return _load().orc_hg_E(self._h)

    @property
    def P(self):
        return _load().orc_hg_P(self._h)

    def arrays(self):
        L = _load()
        off = np.empty(self.E + 1, np.int32)
        pin = np.empty(self.P, np.int32)
        nw = np.empty(self.N, np.int32)
        hw = np.empty(self.E, np.int32)
        L.orc_hg_copy(self._h, _ptr(off), _ptr(pin), _ptr(nw), _ptr(hw))
        return dict(N=self.N, E=self.E, hoff=off, pins=pin, nw=nw, hw=hw)


def hash32(x: int) -> int:
    return int(_load().orc_hash(x & 0xFFFFFFFF))


def priority(g: Hypergraph, e: int, policy) -> int:
    return int(_load().orc_priority(g._h, e, _policy(policy)))


def ceil_sqrt(n: int) -> int:
    return int(_load().orc_ceil_sqrt(n))


def limit(W: int, eps: float) -> int:
    return int(_load().orc_limit(W, eps))


def match(g: Hypergraph, policy) -> np.ndarray:
    out = np.empty(g.N, np.int32)
    _load().orc_match(g._h, _policy(policy), _ptr(out))
    return out


def coarsen_merge(g: Hypergraph, policy):
    """Algorithm 2 followed by reading M1 (parallel nets merged): (coarse, cmap, match)."""
    cm = np.empty(max(g.N, 1), np.int32)
    mt = np.empty(max(g.N, 1), np.int32)
    h = _load().orc_coarsen_ex(g._h, _policy(policy), 1, _ptr(cm), _ptr(mt))
    return Hypergraph(h), cm[: g.N], mt[: g.N]


def merge_parallel(g: Hypergraph) -> "Hypergraph":
    """Reading M1 applied to a copy of g."""
    a = g.arrays()
    h = Hypergraph.from_csr(g.N, a["hoff"], a["pins"], a["nw"], a["hw"])
    _load().orc_merge_parallel(h._h)
    return h


def coarsen(g: Hypergraph, policy):
    """One level of Algorithm 2: returns (coarse Hypergraph, cmap, match)."""
    cmap = np.empty(max(g.N, 1), np.int32)
    m = np.empty(max(g.N, 1), np.int32)
    h = _load().orc_coarsen(g._h, _policy(policy), _ptr(cmap), _ptr(m))
    return Hypergraph(h), cmap[: g.N], m[: g.N]


def gains(g: Hypergraph, side) -> np.ndarray:
    side = np.ascontiguousarray(side, dtype=np.uint8)
    out = np.empty(g.N, np.int32)
    _load().orc_gains(g._h, _ptr(side), _ptr(out))
    return out


def initial(g: Hypergraph, m0=1, m=2):
    """Algorithm 3 with side 0 meant for m0 of m parts (reading G2; 1 of 2 = the paper's)."""
    side = np.empty(max(g.N, 1), np.uint8)
    if (m0, m) == (1, 2):
        rounds = _load().orc_initial(g._h, _ptr(side))
    else:
        rounds = _load().orc_initial_target(g._h, _ptr(side), int(m0), int(m))
    return side[: g.N], int(rounds)


def refine_iter(g: Hypergraph, side: np.ndarray) -> int:
    assert side.dtype == np.uint8 and side.flags.c_contiguous
    return int(_load().orc_refine_iter(g._h, _ptr(side)))


def rebalance(g: Hypergraph, side: np.ndarray, lim: int, lim1=None):
    """Reading C13 (one limit for both sides), or with a limit per side (reading G2)."""
    assert side.dtype == np.uint8 and side.flags.c_contiguous
    rounds = ctypes.c_int32(0)
    if lim1 is None:
        st = _load().orc_rebalance(g._h, _ptr(side), int(lim), ctypes.byref(rounds))
    else:
        st = _load().orc_rebalance2(g._h, _ptr(side), int(lim), int(lim1), ctypes.byref(rounds))
    return int(st), int(rounds.value)


def limit_part(W: int, ms: int, m: int, e6: int) -> int:
    """Reading G2: limit of a side meant for ms of m parts, imbalance e6 millionths."""
    return int(_load().orc_limit_part(int(W), int(ms), int(m), int(e6)))


def adaptive_e6(e6: int, k: int) -> int:
    """Reading G3: per-bisection imbalance (millionths) for k parts."""
    return int(_load().orc_adaptive_e6(int(e6), int(k)))


def bisect(g: Hypergraph, eps=0.1, policy="LDH", levels=25, iters=2, keep_levels=True,
           target=None, e6=None, merge=False):
    """Multilevel bisection: dict(side, status, nlev, init_rounds, limit, levels, cmaps, matches).
    `target` = (m0, m): side 0 meant for m0 of m parts (reading G2); `e6` overrides eps with an
    imbalance in millionths."""
    L = _load()
    if target is None and e6 is None and not merge:
        r = L.orc_bisect(g._h, float(eps), _policy(policy), int(levels), int(iters))
    else:
        m0, m = target if target is not None else (1, 2)
        e = int(e6) if e6 is not None else _e6(eps)
        r = L.orc_bisect_ex(g._h, e, int(m0), int(m), 1 if merge else 0, _policy(policy),
                            int(levels), int(iters))
    try:
        nlev = L.orc_run_nlev(r)
        side = np.empty(max(g.N, 1), np.uint8)
        L.orc_run_side(r, _ptr(side))
        out = dict(side=side[: g.N], status=int(L.orc_run_status(r)), nlev=int(nlev),
                   init_rounds=int(L.orc_run_init_rounds(r)), limit=int(L.orc_run_limit(r)))
        if keep_levels:
            levs, cmaps, matches = [], [], []
            for l in range(nlev):
                h = Hypergraph(L.orc_run_level(r, l), owned=False)
                levs.append(h.arrays())
                if l < nlev - 1:
                    cm = np.empty(max(h.N, 1), np.int32)
                    mt = np.empty(max(h.N, 1), np.int32)
                    L.orc_run_cmap(r, l, _ptr(cm))
                    L.orc_run_match(r, l, _ptr(mt))
                    cmaps.append(cm[: h.N])
                    matches.append(mt[: h.N])
            out.update(levels=levs, cmaps=cmaps, matches=matches)
        return out
    finally:
        L.orc_run_free(r)


def cut(g: Hypergraph, part) -> int:
    part = np.ascontiguousarray(part, dtype=np.int32)
    return int(_load().orc_cut(g._h, _ptr(part)))


def cut_bisection(g: Hypergraph, side) -> int:
    side = np.ascontiguousarray(side, dtype=np.uint8)
    return int(_load().orc_cut_bisection(g._h, _ptr(side)))


def subgraph(g: Hypergraph, part, j: int):
    part = np.ascontiguousarray(part, dtype=np.int32)
    l2g = np.empty(max(g.N, 1), np.int32)
    h = _load().orc_subgraph(g._h, _ptr(part), int(j), _ptr(l2g))
    s = Hypergraph(h)
    return s, l2g[: s.N]


def partition(g: Hypergraph, k=2, eps=0.1, policy="LDH", levels=25, iters=2, adaptive=False,
              merge=False):
    """Nested k-way (Algorithm 6, any k >= 1 by readings G1-G2; `adaptive`: the per-bisection
    imbalance of reading G3; `merge`: parallel nets merged at contraction, reading M1): returns
    (parts int32[N], status)."""
    part = np.empty(max(g.N, 1), np.int32)
    if not adaptive and not merge:
        st = _load().orc_partition(g._h, int(k), float(eps), _policy(policy), int(levels),
                                   int(iters), _ptr(part))
    else:
        flags = (1 if adaptive else 0) | (2 if merge else 0)
        st = _load().orc_partition_ex(g._h, int(k), _e6(eps), flags, _policy(policy),
                                      int(levels), int(iters), _ptr(part))
    return part[: g.N], int(st)
