"""Python binding of libsssp.so, the GB300 library for Garg's bound-based
single-source shortest paths (arXiv 1812.10499).

Argument marshalling only: every function has the name of the C entry point
it calls (include/sssp.h) and every step of the computation runs in the CUDA
kernels of the library.  There is no CPU fallback: if the library has not
been built, load() raises.

PyTorch is used only as plumbing: optional device memory through its caching
allocator (torch_allocator_options) and streams / device tensors for the
_device entry points.
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsssp.so")

SSSP_OK = 0
SSSP_PENDING = 1
SSSP_E_INVAL = -1
SSSP_E_ZERO_WEIGHT = -2
SSSP_E_SOURCE_RANGE = -3
SSSP_E_OVERFLOW = -4
SSSP_E_NOMEM = -5
SSSP_E_DEVICE_TIMEOUT = -6
SSSP_E_CUDA = -7
SSSP_E_ROUND_LIMIT = -8
SSSP_E_BUSY = -9
SSSP_E_NOT_FOUND = -10
SSSP_E_INTERNAL = -11
SSSP_E_NOALLOC_LIMIT = -12
SSSP_RULE_THRESHOLD = 0
SSSP_RULE_MIND = 1
SSSP_RULE_LABEL_CORRECTING = 2
SSSP_RULE_CHEAP_FIRST = 4
SSSP_RULE_WINDOWED = 16
SSSP_RULE_PRED_COUNT = 32
SSSP_LOOP_GRAPH = 0
SSSP_LOOP_HOST = 1
SSSP_LOOP_PERSISTENT = 2
SSSP_SERVE_MANUAL = 1
SSSP_SERVE_WIDE = 2
SSSP_LAYOUT_AUTO = 0
SSSP_LAYOUT_WIDE = 1
SSSP_LAYOUT_COMPACT = 2
SSSP_DIST_INF = 0xFFFFFFFFFFFFFFFF

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class sssp_options(ctypes.Structure):
    _fields_ = [("rule", ctypes.c_uint32), ("loop_mode", ctypes.c_uint32),
                ("hub_degree", ctypes.c_uint32), ("chunk_edges", ctypes.c_uint32),
                ("block_threads", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("device", ctypes.c_int32), ("layout", ctypes.c_uint32),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
                ("delta", ctypes.c_uint64)]


class sssp_solve_args(ctypes.Structure):
    _fields_ = [("dist", ctypes.c_void_p), ("parent", ctypes.c_void_p),
                ("fixed_round", ctypes.c_void_p), ("lower", ctypes.c_void_p),
                ("max_rounds", ctypes.c_uint32), ("dev", ctypes.c_uint32),
                ("cuda_stream", ctypes.c_void_p), ("has_target", ctypes.c_uint32),
                ("target", ctypes.c_uint32)]


class sssp_solve_info(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint32), ("finished", ctypes.c_uint32),
                ("reached", ctypes.c_uint64), ("out_scanned", ctypes.c_uint64),
                ("in_scanned", ctypes.c_uint64), ("active_visits", ctypes.c_uint64),
                ("front_visits", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class sssp_kernel_profile(ctypes.Structure):
    _fields_ = [("relax_launches", ctypes.c_uint64), ("cupdate_launches", ctypes.c_uint64),
                ("relax_ms", ctypes.c_double), ("cupdate_ms", ctypes.c_double),
                ("tail_launches", ctypes.c_uint64), ("tail_ms", ctypes.c_double),
                ("tail_rounds", ctypes.c_uint64), ("grid_counters", ctypes.c_uint64 * 4),
                ("tail_counters", ctypes.c_uint64 * 4)]

    COUNTERS = ("out_scanned", "in_scanned", "active_visits", "front_visits")

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if not k.endswith("counters")}
        d["grid_counters"] = dict(zip(self.COUNTERS, (int(x) for x in self.grid_counters)))
        d["tail_counters"] = dict(zip(self.COUNTERS, (int(x) for x in self.tail_counters)))
        return d


class sssp_serve_cfg(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("max_slots", ctypes.c_uint32),
                ("rounds_per_step", ctypes.c_uint32), ("device", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", ctypes.c_void_p)]


class sssp_query_info(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("submit_ns", ctypes.c_uint64), ("admit_ns", ctypes.c_uint64),
                ("done_ns", ctypes.c_uint64), ("first_step", ctypes.c_uint64),
                ("last_step", ctypes.c_uint64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_ if k != "reserved"}


class sssp_serve_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint64), ("rounds", ctypes.c_uint64),
                ("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("queued", ctypes.c_uint32), ("inflight", ctypes.c_uint32),
                ("max_inflight", ctypes.c_uint32), ("layout", ctypes.c_uint32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class sssp_tuning(ctypes.Structure):
    _fields_ = [("hub_degree", ctypes.c_uint32), ("chunk_edges", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("tail_items", ctypes.c_uint32)]

    FIELDS = ("hub_degree", "chunk_edges", "ctas_per_sm", "tail_items")

    def as_dict(self):
        return {k: int(getattr(self, k)) for k in self.FIELDS}

    @classmethod
    def from_dict(cls, d):
        t = cls()
        for k in cls.FIELDS:
            setattr(t, k, int(d[k]))
        return t


class sssp_tune_result(ctypes.Structure):
    _fields_ = [("best", sssp_tuning), ("start_ms", ctypes.c_double),
                ("best_ms", ctypes.c_double), ("evaluated", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]

    def as_dict(self):
        return {"best": self.best.as_dict(), "start_ms": self.start_ms, "best_ms": self.best_ms,
                "evaluated": int(self.evaluated)}


class SsspError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {sssp_strerror(code)} ({code})")


_lib = None
# ctypes callbacks must outlive the handles that use them.
_keepalive: dict = {}


def load(path: str = LIB_PATH):
    """Loads libsssp.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, u32, u64, i32, c_int = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                ctypes.c_int32, ctypes.c_int)
    sig = {
        "sssp_options_default": (None, [ctypes.POINTER(sssp_options)]),
        "sssp_create": (c_int, [u32, u64, vp, vp, vp, vp, vp, vp,
                                ctypes.POINTER(sssp_options), ctypes.POINTER(vp)]),
        "sssp_solve": (c_int, [vp, u32, vp, ctypes.POINTER(u32)]),
        "sssp_solve_device": (c_int, [vp, u32, vp, ctypes.POINTER(u32), vp]),
        "sssp_solve_ex": (c_int, [vp, u32, ctypes.POINTER(sssp_solve_args),
                                  ctypes.POINTER(sssp_solve_info)]),
        "sssp_solve_batch": (c_int, [vp, vp, u32, vp, vp]),
        "sssp_solve_batch_device": (c_int, [vp, vp, u32, vp, vp, vp]),
        "sssp_serve_open": (c_int, [ctypes.POINTER(sssp_serve_cfg), ctypes.POINTER(vp)]),
        "sssp_serve_submit": (c_int, [vp, vp, u32, vp, ctypes.POINTER(u64)]),
        "sssp_serve_poll": (c_int, [vp, u64, ctypes.POINTER(u32)]),
        "sssp_serve_wait": (c_int, [vp, u64, u32, ctypes.POINTER(sssp_query_info)]),
        "sssp_serve_stats_get": (c_int, [vp, ctypes.POINTER(sssp_serve_stats)]),
        "sssp_serve_drain": (c_int, [vp]),
        "sssp_serve_close": (None, [vp]),
        "sssp_profile": (c_int, [vp, c_int, ctypes.POINTER(sssp_kernel_profile)]),
        "sssp_profile_rounds": (c_int, [vp, vp, vp, vp, vp, vp, u32, ctypes.POINTER(u32)]),
        "sssp_solve_noalloc": (c_int, [u32, vp, vp, vp, vp, u32, u32, vp,
                                       ctypes.POINTER(u32), vp]),
        "sssp_get_tuning": (c_int, [vp, ctypes.POINTER(sssp_tuning)]),
        "sssp_set_tuning": (c_int, [vp, ctypes.POINTER(sssp_tuning)]),
        "sssp_tune_key": (c_int, [u32, u64, u32, u32, u32, ctypes.c_char_p, ctypes.c_size_t]),
        "sssp_graph_key": (c_int, [vp, ctypes.c_char_p, ctypes.c_size_t]),
        "sssp_batch_key": (c_int, [vp, u32, ctypes.c_char_p, ctypes.c_size_t]),
        "sssp_tune_cache_open": (c_int, [ctypes.c_char_p]),
        "sssp_tune_cache_get": (c_int, [ctypes.c_char_p, ctypes.POINTER(sssp_tuning)]),
        "sssp_tune_cache_put": (c_int, [ctypes.c_char_p, ctypes.POINTER(sssp_tuning)]),
        "sssp_autotune": (c_int, [vp, vp, u32, u32, ctypes.POINTER(sssp_tune_result)]),
        "sssp_autotune_batch": (c_int, [vp, vp, u32, u32, ctypes.POINTER(sssp_tune_result)]),
        "sssp_destroy": (None, [vp]),
        "sssp_host_alloc": (c_int, [ctypes.c_size_t, ctypes.POINTER(vp)]),
        "sssp_host_free": (None, [vp]),
        "sssp_strerror": (ctypes.c_char_p, [c_int]),
        "sssp_num_vertices": (u32, [vp]),
        "sssp_num_edges": (u64, [vp]),
        "sssp_layout": (u32, [vp]),
        "sssp_selftest_barrier_timeout": (c_int, [u32]),
        "sssp_solve_to": (c_int, [vp, u32, u32, ctypes.POINTER(u64), ctypes.POINTER(u32)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, what: str):
    if rc != SSSP_OK:
        raise SsspError(rc, what)


def _ptr(a):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def sssp_strerror(code: int) -> str:
    return load().sssp_strerror(code).decode()


def sssp_options_default() -> sssp_options:
    o = sssp_options()
    load().sssp_options_default(ctypes.byref(o))
    return o


def torch_allocator_options(opt: sssp_options | None = None, device: int | None = None):
    """Options whose allocator hooks take device memory from PyTorch's CUDA
    caching allocator."""
    import torch

    opt = opt or sssp_options_default()
    dev = torch.cuda.current_device() if device is None else device

    def _alloc(nbytes, _ctx):
        return torch.cuda.caching_allocator_alloc(int(nbytes), device=dev)

    def _free(ptr, _ctx):
        torch.cuda.caching_allocator_delete(ptr)

    opt.alloc = ALLOC_FN(_alloc)
    opt.free = FREE_FN(_free)
    opt.device = dev
    _keepalive[id(opt)] = (opt.alloc, opt.free)
    return opt


def _contig(a, dtype):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=dtype)


def sssp_create(n: int, row_ptr, col, w, col_ptr=None, row=None, w_in=None,
                options: sssp_options | None = None) -> int:
    """Device-resident graph from a host CSR (and optional CSC); returns the handle."""
    lib = load()
    row_ptr = _contig(row_ptr, np.uint64)
    col, w = _contig(col, np.uint32), _contig(w, np.uint32)
    col_ptr, row, w_in = _contig(col_ptr, np.uint64), _contig(row, np.uint32), _contig(w_in, np.uint32)
    m = int(row_ptr[-1]) if row_ptr is not None and len(row_ptr) else 0
    if row_ptr is None or len(row_ptr) != n + 1 or len(col) != m or len(w) != m:
        raise SsspError(-1, "sssp_create")
    h = ctypes.c_void_p()
    rc = lib.sssp_create(n, m, _ptr(row_ptr), _ptr(col) if m else None, _ptr(w) if m else None,
                         _ptr(col_ptr), _ptr(row) if row is not None and m else None,
                         _ptr(w_in) if w_in is not None and m else None,
                         ctypes.byref(options) if options is not None else None, ctypes.byref(h))
    _check(rc, "sssp_create")
    if options is not None and id(options) in _keepalive:
        _keepalive[h.value] = _keepalive[id(options)]
    return h.value


def sssp_destroy(h: int):
    if h:
        load().sssp_destroy(h)
        _keepalive.pop(h, None)


def host_empty(n: int, dtype=np.uint64) -> np.ndarray:
    """An uninitialised numpy array of n elements in page-locked host memory
    (sssp_host_alloc), freed when the array is collected.  Passed as the
    `out` of sssp_solve it takes the distances by DMA every solve."""
    lib = load()
    dt = np.dtype(dtype)
    nbytes = max(1, int(n) * dt.itemsize)
    p = ctypes.c_void_p()
    _check(lib.sssp_host_alloc(nbytes, ctypes.byref(p)), "sssp_host_alloc")
    buf = (ctypes.c_char * nbytes).from_address(p.value)
    weakref.finalize(buf, lib.sssp_host_free, p.value)
    return np.frombuffer(buf, dtype=dt, count=int(n))


def sssp_profile(h: int, enable: bool) -> dict:
    """Switches per-kernel CUDA-event timing on or off; returns (and resets)
    the totals gathered so far."""
    p = sssp_kernel_profile()
    _check(load().sssp_profile(h, int(bool(enable)), ctypes.byref(p)), "sssp_profile")
    return p.as_dict()


def sssp_profile_rounds(h: int):
    """Per-iteration (relax_ms, cupdate_ms, tail_ms, tail_rounds, counters)
    arrays of the last profiled solve; counters is u64[iterations, 4]:
    out_scanned, in_scanned, active_visits, front_visits of the iteration's
    k_relax and k_cupdate (device-loop schedule only)."""
    lib = load()
    cnt = ctypes.c_uint32(0)
    _check(lib.sssp_profile_rounds(h, None, None, None, None, None, 0, ctypes.byref(cnt)),
           "sssp_profile_rounds")
    r = np.zeros(cnt.value, dtype=np.float32)
    c = np.zeros(cnt.value, dtype=np.float32)
    t = np.zeros(cnt.value, dtype=np.float32)
    tr = np.zeros(cnt.value, dtype=np.uint32)
    ctr = np.zeros((cnt.value, 4), dtype=np.uint64)
    _check(lib.sssp_profile_rounds(h, r.ctypes.data, c.ctypes.data, t.ctypes.data,
                                   tr.ctypes.data, ctr.ctypes.data, cnt.value,
                                   ctypes.byref(cnt)),
           "sssp_profile_rounds")
    return r, c, t, tr, ctr


def sssp_solve_noalloc(n: int, out_off, out_adj, in_off, in_adj, source: int, max_weight: int,
                       dist_dev, stream=None) -> int:
    """Solve for callers that cannot allocate device memory: the graph
    (out_off u64[n+1], out_adj (target, weight) u32 pairs, and the same by
    target) and dist_dev are the caller's CUDA tensors; the library uses only
    its fixed scratch.  Returns the round count."""
    r = ctypes.c_uint32(0)
    _check(load().sssp_solve_noalloc(n, _ptr(out_off), _ptr(out_adj), _ptr(in_off),
                                     _ptr(in_adj), source, max_weight, _ptr(dist_dev),
                                     ctypes.byref(r), _stream_ptr(stream)),
           "sssp_solve_noalloc")
    return int(r.value)


def sssp_num_vertices(h: int) -> int:
    return load().sssp_num_vertices(h)


def sssp_num_edges(h: int) -> int:
    return load().sssp_num_edges(h)


def sssp_solve_to(h: int, source: int, target: int):
    """Single-target query: (cost[target] or SSSP_DIST_INF, rounds executed)."""
    d = ctypes.c_uint64(0)
    r = ctypes.c_uint32(0)
    _check(load().sssp_solve_to(h, source, target, ctypes.byref(d), ctypes.byref(r)),
           "sssp_solve_to")
    return int(d.value), int(r.value)


def sssp_selftest_barrier_timeout(timeout_ms: int = 200) -> int:
    """Status of the device-wait self-test (SSSP_E_DEVICE_TIMEOUT = -6 when the
    wait limit worked)."""
    return load().sssp_selftest_barrier_timeout(timeout_ms)


def sssp_layout(h: int) -> int:
    """SSSP_LAYOUT_WIDE or SSSP_LAYOUT_COMPACT: the handle's state layout."""
    return load().sssp_layout(h)


def sssp_solve(h: int, source: int, out: np.ndarray | None = None):
    """Returns (dist u64[n], rounds).  out: a C-contiguous u64[n] array to
    write the distances into (reused across calls, it saves allocating and
    first-touching n * 8 bytes of host memory per call)."""
    lib = load()
    n = lib.sssp_num_vertices(h)
    if out is None:
        dist = np.empty(n, dtype=np.uint64)
    else:
        if out.dtype != np.uint64 or out.shape != (n,) or not out.flags.c_contiguous:
            raise SsspError(-1, "sssp_solve: out must be a contiguous u64[n] array")
        dist = out
    rounds = ctypes.c_uint32(0)
    _check(lib.sssp_solve(h, source, _ptr(dist), ctypes.byref(rounds)), "sssp_solve")
    return dist, int(rounds.value)


def sssp_solve_device(h: int, source: int, dist_dev, stream=None, want_rounds: bool = False):
    """dist_dev: a CUDA tensor (u64/int64, n entries).  Enqueues on `stream`
    (a torch.cuda.Stream or raw handle); returns the round count only if
    want_rounds (which synchronises)."""
    lib = load()
    rounds = ctypes.c_uint32(0)
    rc = lib.sssp_solve_device(h, source, _ptr(dist_dev),
                               ctypes.byref(rounds) if want_rounds else None, _stream_ptr(stream))
    _check(rc, "sssp_solve_device")
    return int(rounds.value) if want_rounds else None


def sssp_solve_ex(h: int, source: int, *, dist=True, parent=False, fixed_round=False,
                  lower=False, max_rounds: int = 0, stream=None, target: int | None = None) -> dict:
    """Host outputs chosen by flag, plus the solve counters."""
    lib = load()
    n = lib.sssp_num_vertices(h)
    out = {}
    a = sssp_solve_args()
    if dist:
        out["dist"] = np.empty(n, dtype=np.uint64)
        a.dist = out["dist"].ctypes.data
    if parent:
        out["parent"] = np.empty(n, dtype=np.uint32)
        a.parent = out["parent"].ctypes.data
    if fixed_round:
        out["fixed_round"] = np.empty(n, dtype=np.int32)
        a.fixed_round = out["fixed_round"].ctypes.data
    if lower:
        out["lower"] = np.empty(n, dtype=np.uint64)
        a.lower = out["lower"].ctypes.data
    a.max_rounds = max_rounds
    a.has_target = 0 if target is None else 1
    a.target = 0 if target is None else int(target)
    a.dev = 0
    a.cuda_stream = _stream_ptr(stream)
    info = sssp_solve_info()
    _check(lib.sssp_solve_ex(h, source, ctypes.byref(a), ctypes.byref(info)), "sssp_solve_ex")
    out["info"] = info.as_dict()
    return out


def _handle_array(handles):
    arr = (ctypes.c_void_p * len(handles))(*handles)
    return arr


def sssp_solve_batch(handles, sources):
    """k queries in one lock-step launch; returns (list of dist arrays, rounds u32[k])."""
    lib = load()
    k = len(handles)
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    dists = [np.empty(lib.sssp_num_vertices(h), dtype=np.uint64) for h in handles]
    ptrs = (ctypes.c_void_p * k)(*[d.ctypes.data for d in dists])
    rounds = np.zeros(k, dtype=np.uint32)
    _check(lib.sssp_solve_batch(_handle_array(handles), src.ctypes.data, k, ptrs,
                                rounds.ctypes.data), "sssp_solve_batch")
    return dists, rounds


def sssp_solve_batch_device(handles, sources, dist_devs, stream=None):
    """Device-output form; dist_devs are CUDA tensors.  Returns rounds u32[k]."""
    lib = load()
    k = len(handles)
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    ptrs = (ctypes.c_void_p * k)(*[_ptr(d) for d in dist_devs])
    rounds = np.zeros(k, dtype=np.uint32)
    _check(lib.sssp_solve_batch_device(_handle_array(handles), src.ctypes.data, k, ptrs,
                                       rounds.ctypes.data, _stream_ptr(stream)),
           "sssp_solve_batch_device")
    return rounds


def sssp_serve_open(budget_bytes: int = 0, max_slots: int = 0, rounds_per_step: int = 0,
                    device: int = -1, flags: int = 0) -> int:
    """Opens a server; flags: SSSP_SERVE_MANUAL (no server thread: poll,
    wait and drain run the steps), SSSP_SERVE_WIDE (32-byte records)."""
    cfg = sssp_serve_cfg()
    cfg.budget_bytes = budget_bytes
    cfg.max_slots = max_slots
    cfg.rounds_per_step = rounds_per_step
    cfg.device = device
    cfg.flags = flags
    s = ctypes.c_void_p()
    _check(load().sssp_serve_open(ctypes.byref(cfg), ctypes.byref(s)), "sssp_serve_open")
    return s.value


def sssp_serve_submit(server: int, h: int, source: int, dist_out: np.ndarray) -> int:
    """Queues a query; dist_out (u64[n], host) is written when it completes."""
    t = ctypes.c_uint64(0)
    _check(load().sssp_serve_submit(server, h, source, dist_out.ctypes.data, ctypes.byref(t)),
           "sssp_serve_submit")
    return int(t.value)


def sssp_serve_poll(server: int, ticket: int):
    """Returns (status, rounds): status SSSP_OK when done, SSSP_PENDING otherwise."""
    r = ctypes.c_uint32(0)
    rc = load().sssp_serve_poll(server, ticket, ctypes.byref(r))
    if rc not in (SSSP_OK, SSSP_PENDING):
        raise SsspError(rc, "sssp_serve_poll")
    return rc, int(r.value)


def sssp_serve_wait(server: int, ticket: int, timeout_ms: int):
    """Waits up to timeout_ms; returns (status, info dict or None): status
    SSSP_OK with the query's rounds and monotonic-clock times (ns), or
    SSSP_PENDING when the time ran out."""
    info = sssp_query_info()
    rc = load().sssp_serve_wait(server, ticket, timeout_ms, ctypes.byref(info))
    if rc not in (SSSP_OK, SSSP_PENDING):
        raise SsspError(rc, "sssp_serve_wait")
    return rc, (info.as_dict() if rc == SSSP_OK else None)


def sssp_serve_stats_get(server: int) -> dict:
    st = sssp_serve_stats()
    _check(load().sssp_serve_stats_get(server, ctypes.byref(st)), "sssp_serve_stats_get")
    return st.as_dict()


def sssp_serve_drain(server: int):
    _check(load().sssp_serve_drain(server), "sssp_serve_drain")


def sssp_serve_close(server: int):
    if server:
        load().sssp_serve_close(server)


# ----------------------------------------------------------------- tuning

def sssp_get_tuning(h: int) -> dict:
    t = sssp_tuning()
    _check(load().sssp_get_tuning(h, ctypes.byref(t)), "sssp_get_tuning")
    return t.as_dict()


def sssp_set_tuning(h: int, tuning: dict):
    t = sssp_tuning.from_dict(tuning)
    _check(load().sssp_set_tuning(h, ctypes.byref(t)), "sssp_set_tuning")


def sssp_tune_key(n: int, m: int, max_out: int, max_in: int, max_weight: int) -> str:
    buf = ctypes.create_string_buffer(96)
    _check(load().sssp_tune_key(n, m, max_out, max_in, max_weight, buf, 96), "sssp_tune_key")
    return buf.value.decode()


def sssp_graph_key(h: int) -> str:
    buf = ctypes.create_string_buffer(96)
    _check(load().sssp_graph_key(h, buf, 96), "sssp_graph_key")
    return buf.value.decode()


def sssp_batch_key(handles) -> str:
    buf = ctypes.create_string_buffer(96)
    _check(load().sssp_batch_key(_handle_array(handles), len(handles), buf, 96), "sssp_batch_key")
    return buf.value.decode()


def sssp_tune_cache_open(path: str | None):
    _check(load().sssp_tune_cache_open(None if path is None else path.encode()),
           "sssp_tune_cache_open")


def sssp_tune_cache_get(key: str) -> dict | None:
    t = sssp_tuning()
    rc = load().sssp_tune_cache_get(key.encode(), ctypes.byref(t))
    if rc == SSSP_E_NOT_FOUND:
        return None
    _check(rc, "sssp_tune_cache_get")
    return t.as_dict()


def sssp_tune_cache_put(key: str, tuning: dict):
    t = sssp_tuning.from_dict(tuning)
    _check(load().sssp_tune_cache_put(key.encode(), ctypes.byref(t)), "sssp_tune_cache_put")


def sssp_autotune(h: int, sources, reps: int = 0) -> dict:
    """Times candidate tunings on the device, sets the fastest on the handle
    and caches it under the graph's class; returns the sweep's result."""
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    r = sssp_tune_result()
    _check(load().sssp_autotune(h, src.ctypes.data, len(src), reps, ctypes.byref(r)),
           "sssp_autotune")
    return r.as_dict()


def sssp_autotune_batch(handles, sources, reps: int = 0) -> dict:
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    r = sssp_tune_result()
    _check(load().sssp_autotune_batch(_handle_array(handles), src.ctypes.data, len(handles),
                                      reps, ctypes.byref(r)), "sssp_autotune_batch")
    return r.as_dict()
