"""Python binding of the GB300 BiPart library (``libbipart.so``, C ABI in include/bipart.h).

Argument marshalling only: every step of the partitioner runs in the library's sm_103a kernels.
PyTorch supplies device memory (its caching allocator backs every buffer the library allocates)
and streams (calls run on ``torch.cuda.current_stream()`` unless a stream is given).  There is
no CPU fallback: if the CUDA library cannot be built or loaded, or no GPU is present, calls raise.

Names follow the C ABI: ``create`` / ``create_device`` -> :class:`Handle`, and on a handle
``partition``, ``partition_device``, ``num_levels``, ``get_level``, ``cut``, ``sizes``.
"""
from __future__ import annotations

import atexit
import ctypes
import threading
import weakref

import numpy as np

from . import _build

OK = 0
WARN_IMBALANCED = 1
ERR_INVALID_ARG = -1
ERR_INVALID_CSR = -2
ERR_OOM = -3
ERR_CUDA = -4
ERR_TIMEOUT = -5

POLICIES = {"LDH": 0, "HDH": 1, "LWD": 2, "HWD": 3, "RAND": 4}

_lock = threading.Lock()
_lib = None
_handles = weakref.WeakSet()
_alloc_cb = None
_free_cb = None

_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_p32 = ctypes.POINTER(ctypes.c_int32)
class Instance(ctypes.Structure):
    _fields_ = [("num_nodes", ctypes.c_int32), ("num_hedges", ctypes.c_int32),
                ("hedge_offsets", ctypes.c_void_p), ("hedge_pins", ctypes.c_void_p),
                ("node_weights", ctypes.c_void_p), ("hedge_weights", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("epsilon", ctypes.c_double), ("policy", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("refine_iters", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


FLAG_ADAPTIVE_EPS = 1
FLAG_MERGE_PARALLEL = 2


_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)

SYMBOLS = {
    "bipart_set_allocator": (ctypes.c_int, [_ALLOC, _FREE, _vp]),
    "bipart_create": (ctypes.c_int, [_i32, _i32, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "bipart_create_device": (ctypes.c_int, [_i32, _i32, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "bipart_set_stream": (ctypes.c_int, [_vp, _vp]),
    "bipart_partition": (ctypes.c_int, [_vp, _i32, ctypes.c_double, _i32, _i32, _i32, _vp]),
    "bipart_partition_device": (ctypes.c_int, [_vp, _i32, ctypes.c_double, _i32, _i32, _i32, _vp]),
    "bipart_partition_ex": (ctypes.c_int, [_vp, _vp, _vp]),
    "bipart_plan_active": (ctypes.c_int, [_vp, _vp]),
    "bipart_refine_kept": (ctypes.c_int, [_vp, ctypes.c_double, _i32, _vp]),
    "bipart_partition_device_ex": (ctypes.c_int, [_vp, _vp, _vp]),
    "bipart_num_levels": (ctypes.c_int, [_vp, _p32]),
    "bipart_get_level": (ctypes.c_int, [_vp, _i32, _p32, _p32, _p32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "bipart_cut": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(ctypes.c_int64)]),
    "bipart_sizes": (ctypes.c_int, [_vp, _p32, _p32, _p32]),
    "bipart_destroy": (None, [_vp]),
    "bipart_last_error": (ctypes.c_char_p, []),
    "bipart_cut_noalloc": (ctypes.c_int, [_i32, _i32, _vp, _vp, _vp, _vp, _i32, _vp, _vp]),
    "bipart_partition_batch": (ctypes.c_int, [_i32, _vp, _vp, _vp, _vp, _i32]),
    "bipart_batch_tune": (ctypes.c_int, [_i32, _vp, _vp, _vp]),
    "bipart_batch_release": (None, []),
    "bipart_server_create": (ctypes.c_int, [ctypes.c_size_t, _i32, ctypes.POINTER(_vp)]),
    "bipart_server_submit": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_int64)]),
    "bipart_server_wait": (ctypes.c_int, [_vp, ctypes.c_int64, _i32, _p32,
                                          ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]),
    "bipart_server_destroy": (None, [_vp]),
    "bipart_server_stats": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "bipart_kernel_launches": (ctypes.c_int64, []),
    "bipart_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "bipart_profile_select": (ctypes.c_int, [ctypes.c_char_p]),
    "bipart_profile_read": (ctypes.c_int, [_i32, ctypes.c_char_p, ctypes.c_size_t,
                                           ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double)]),
}


class BipartError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"bipart error {code}: {msg}")
        self.code = code


def build(force: bool = False) -> str:
    """Compiles libbipart.so for sm_103a (in-tree)."""
    return _build.build(force=force)


def load(build_if_needed: bool = True):
    """Loads the CUDA library (building it first if needed) and declares its symbols."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_needed else _build.LIB
            lib = ctypes.CDLL(path)
            for name, (res, args) in SYMBOLS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _check(code):
    if code < 0:
        raise BipartError(code, load().bipart_last_error().decode())
    return code


def use_torch_allocator():
    """Routes the library's device allocations through PyTorch's caching allocator.  The hooks
    are Python callbacks: each allocation takes the interpreter lock, which serialises the
    library's own host threads (batch, server, nested k-way) while it is set."""
    global _alloc_cb, _free_cb
    import torch

    def _alloc(ctx, nbytes, stream):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                          int(stream or 0)))
        except Exception:
            return None

    def _free(ctx, ptr, nbytes, stream):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    _alloc_cb, _free_cb = _ALLOC(_alloc), _FREE(_free)
    _check(load().bipart_set_allocator(_alloc_cb, _free_cb, None))


def use_default_allocator():
    """Restores the library's own allocator (cudaMallocAsync on the handle's stream).  Buffers
    made by another allocator are still returned to it."""
    _check(load().bipart_set_allocator(_ALLOC(), _FREE(), None))


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().bipart_kernel_launches())


def profile_enable(on=True):
    """Per-kernel timing on (True / 1), per kernel and level ("levels" / 2), or off."""
    mode = 2 if on in ("levels", 2) else (1 if on else 0)
    _check(load().bipart_profile_enable(mode))


def profile_select(name=None):
    """Time only the kernel `name` (None: all)."""
    _check(load().bipart_profile_select(name.encode() if name else None))


def profile_read() -> dict:
    """Per-kernel totals: {name: (launches, total_ms, total_algorithmic_bytes)}."""
    L = load()
    n = L.bipart_profile_read(-1, None, 0, None, None, None)
    out = {}
    for i in range(n):
        name = ctypes.create_string_buffer(64)
        cnt, ms, by = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        _check(L.bipart_profile_read(i, name, 64, ctypes.byref(cnt), ctypes.byref(ms), ctypes.byref(by)))
        out[name.value.decode()] = (cnt.value, ms.value, by.value)
    return out


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _np32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _policy(p):
    return POLICIES[p] if isinstance(p, str) else int(p)


class Handle:
    """A hypergraph resident on the GPU (level 0 built), see bipart_create."""

    def __init__(self, raw):
        self._h = raw
        _handles.add(self)

    def close(self):
        if self._h:
            load().bipart_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sizes(self):
        N, E, P = _i32(), _i32(), _i32()
        _check(load().bipart_sizes(self._h, ctypes.byref(N), ctypes.byref(E), ctypes.byref(P)))
        return N.value, E.value, P.value

    def set_stream(self, stream):
        _check(load().bipart_set_stream(self._h, _stream_ptr(stream)))

    def partition(self, k=2, eps=0.1, policy="LDH", levels=25, iters=2, adaptive_eps=False,
                  merge_parallel=False):
        """Returns (parts int32[N] on the host, status).  Any k >= 1; `adaptive_eps` gives every
        bisection of a k-way partition the per-bisection imbalance (BIPART_FLAG_ADAPTIVE_EPS);
        `merge_parallel` merges parallel nets at contraction (BIPART_FLAG_MERGE_PARALLEL)."""
        N = self.sizes()[0]
        out = np.empty(max(N, 1), np.int32)
        if adaptive_eps or merge_parallel:
            p = _params(k, eps, policy, levels, iters, adaptive_eps, merge_parallel)
            st = _check(load().bipart_partition_ex(self._h, ctypes.byref(p), _ptr(out)))
        else:
            st = _check(load().bipart_partition(self._h, int(k), float(eps), _policy(policy),
                                                int(levels), int(iters), _ptr(out)))
        return out[:N], st

    def partition_device(self, out, k=2, eps=0.1, policy="LDH", levels=25, iters=2,
                         adaptive_eps=False, merge_parallel=False):
        """Writes parts into the int32 CUDA tensor `out` (asynchronously on the handle's stream)."""
        if adaptive_eps or merge_parallel:
            p = _params(k, eps, policy, levels, iters, adaptive_eps, merge_parallel)
            return _check(load().bipart_partition_device_ex(self._h, ctypes.byref(p),
                                                            ctypes.c_void_p(out.data_ptr())))
        return _check(load().bipart_partition_device(self._h, int(k), float(eps), _policy(policy),
                                                     int(levels), int(iters),
                                                     ctypes.c_void_p(out.data_ptr())))

    def refine_kept(self, eps=0.1, iters=2):
        """bipart_refine_kept: Algorithm 3 and the refinement again on the hierarchy of the last
        k = 2 partition, with a new imbalance and iteration count.  Returns (parts, status)."""
        N = self.sizes()[0]
        out = np.empty(max(N, 1), np.int32)
        st = _check(load().bipart_refine_kept(self._h, float(eps), int(iters), _ptr(out)))
        return out[:N], st

    def plan_active(self) -> bool:
        """Whether the last partition call replayed a captured CUDA graph (diagnostics)."""
        a = _i32()
        _check(load().bipart_plan_active(self._h, ctypes.byref(a)))
        return bool(a.value)

    def num_levels(self):
        n = _i32()
        _check(load().bipart_num_levels(self._h, ctypes.byref(n)))
        return n.value

    def get_level(self, level):
        L = load()
        N, E, P = _i32(), _i32(), _i32()
        _check(L.bipart_get_level(self._h, int(level), ctypes.byref(N), ctypes.byref(E),
                                  ctypes.byref(P), None, None, None, None, None, None))
        n, e, p = N.value, E.value, P.value
        hoff = np.empty(e + 1, np.int32)
        pins = np.empty(max(p, 1), np.int32)
        nw = np.empty(max(n, 1), np.int32)
        hw = np.empty(max(e, 1), np.int32)
        cmap = np.empty(max(n, 1), np.int32)
        match = np.empty(max(n, 1), np.int32)
        _check(L.bipart_get_level(self._h, int(level), ctypes.byref(N), ctypes.byref(E),
                                  ctypes.byref(P), _ptr(hoff), _ptr(pins), _ptr(nw), _ptr(hw),
                                  _ptr(cmap), _ptr(match)))
        return dict(N=n, E=e, P=p, hoff=hoff, pins=pins[:p], nw=nw[:n], hw=hw[:e],
                    cmap=cmap[:n], match=match[:n])

    def cut(self, parts):
        parts = _np32(parts)
        c = ctypes.c_int64()
        _check(load().bipart_cut(self._h, _ptr(parts), ctypes.byref(c)))
        return c.value


def create(N, hoff, pins, nw=None, hw=None, stream=None) -> Handle:
    """bipart_create on host arrays."""
    L = load()
    hoff, pins, nw, hw = _np32(hoff), _np32(pins), _np32(nw), _np32(hw)
    out = ctypes.c_void_p()
    _check(L.bipart_create(int(N), int(hoff.size - 1), _ptr(hoff), _ptr(pins), _ptr(nw), _ptr(hw),
                           _stream_ptr(stream), ctypes.byref(out)))
    return Handle(out)


def create_device(N, hoff, pins, nw=None, hw=None, stream=None) -> Handle:
    """bipart_create_device on int32 CUDA tensors."""
    L = load()
    out = ctypes.c_void_p()

    def dp(t):
        return None if t is None else ctypes.c_void_p(t.data_ptr())

    _check(L.bipart_create_device(int(N), int(hoff.numel() - 1), dp(hoff), dp(pins), dp(nw), dp(hw),
                                  _stream_ptr(stream), ctypes.byref(out)))
    return Handle(out)


def cut_noalloc(N, hoff, pins, hw, parts, k, out, stream=None) -> int:
    """bipart_cut_noalloc on CUDA tensors: writes the cut into the int64 tensor `out` (one element)
    without any device allocation by the library; returns the status code."""

    def dp(t):
        return None if t is None else ctypes.c_void_p(t.data_ptr())

    return _check(load().bipart_cut_noalloc(int(N), int(hoff.numel() - 1), dp(hoff), dp(pins),
                                            dp(hw), dp(parts), int(k), dp(out), _stream_ptr(stream)))


def create_from(g: dict, stream=None) -> Handle:
    return create(g["N"], g["hoff"], g["pins"], g.get("nw"), g.get("hw"), stream=stream)


def _instance(g):
    """Instance struct + the arrays it points to (kept alive by the caller)."""
    arrs = [_np32(g["hoff"]), _np32(g["pins"]), _np32(g.get("nw")), _np32(g.get("hw"))]
    inst = Instance(int(g["N"]), int(arrs[0].size - 1), *[_ptr(a) for a in arrs])
    return inst, arrs


def _params(k=2, eps=0.1, policy="LDH", levels=25, iters=2, adaptive_eps=False,
            merge_parallel=False):
    return Params(int(k), float(eps), _policy(policy), int(levels), int(iters),
                  (FLAG_ADAPTIVE_EPS if adaptive_eps else 0) |
                  (FLAG_MERGE_PARALLEL if merge_parallel else 0))


def _batch_args(graphs, params):
    n = len(graphs)
    if isinstance(params, dict):
        params = [params] * n
    keep, insts = [], (Instance * max(n, 1))()
    pars = (Params * max(n, 1))()
    for i, g in enumerate(graphs):
        inst, arrs = _instance(g)
        keep.append(arrs)
        insts[i] = inst
        pars[i] = _params(**params[i])
    return n, keep, insts, pars


def partition_batch(graphs, params, workers=0):
    """bipart_partition_batch: graphs = list of dicts (N, hoff, pins, nw, hw), params = list of
    dicts (k, eps, policy, levels, iters) or one dict for all.  Returns (parts list, statuses)."""
    n, keep, insts, pars = _batch_args(graphs, params)
    outs = [np.empty(max(int(g["N"]), 1), np.int32) for g in graphs]
    out_ptrs = (ctypes.c_void_p * max(n, 1))(*[o.ctypes.data for o in outs])
    st = np.zeros(max(n, 1), np.int32)
    _check(load().bipart_partition_batch(n, ctypes.cast(insts, ctypes.c_void_p),
                                         ctypes.cast(pars, ctypes.c_void_p),
                                         ctypes.cast(out_ptrs, ctypes.c_void_p), _ptr(st), int(workers)))
    return [o[: int(g["N"])] for o, g in zip(outs, graphs)], st[:n]


def tune_batch(graphs, params):
    """bipart_batch_tune: times every block shape on each size bucket of this batch and records
    the fastest (in the JSON tuning cache).  Returns {bucket: (threads, blocks per SM)} for the
    buckets the batch has instances in."""
    n, keep, insts, pars = _batch_args(graphs, params)
    chosen = np.zeros(8, np.int32)
    _check(load().bipart_batch_tune(n, ctypes.cast(insts, ctypes.c_void_p), ctypes.cast(pars, ctypes.c_void_p),
                                    _ptr(chosen)))
    return {b: (int(chosen[2 * b]), int(chosen[2 * b + 1])) for b in range(4) if chosen[2 * b]}


def batch_release():
    """bipart_batch_release: frees the buffers the batch path keeps between calls."""
    load().bipart_batch_release()


class Server:
    """bipart_server_*: submit(graph, params) -> ticket; wait(ticket) -> (parts, status, queue_ms,
    run_ms).  Input arrays and the output buffer are kept alive here until waited for."""

    def __init__(self, hbm_budget_bytes=0, workers=8):
        h = ctypes.c_void_p()
        _check(load().bipart_server_create(int(hbm_budget_bytes), int(workers), ctypes.byref(h)))
        self._h = h
        self._live = {}

    def submit(self, g, **params):
        inst, arrs = _instance(g)
        par = _params(**params)
        out = np.empty(max(int(g["N"]), 1), np.int32)
        t = ctypes.c_int64()
        _check(load().bipart_server_submit(self._h, ctypes.byref(inst), ctypes.byref(par),
                                           _ptr(out), ctypes.byref(t)))
        self._live[t.value] = (inst, arrs, par, out, int(g["N"]))
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        st = _i32()
        qms, rms = ctypes.c_double(), ctypes.c_double()
        _check(load().bipart_server_wait(self._h, int(ticket), int(timeout_ms), ctypes.byref(st),
                                         ctypes.byref(qms), ctypes.byref(rms)))
        inst, arrs, par, out, n = self._live.pop(ticket)
        return out[:n], st.value, qms.value, rms.value

    def stats(self):
        """(micro-batches run, requests they held) so far."""
        b, r = ctypes.c_int64(), ctypes.c_int64()
        _check(load().bipart_server_stats(self._h, ctypes.byref(b), ctypes.byref(r)))
        return int(b.value), int(r.value)

    def close(self):
        if self._h:
            load().bipart_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


@atexit.register
def _close_all():
    for h in list(_handles):
        try:
            h.close()
        except Exception:
            pass
