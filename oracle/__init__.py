"""CPU oracle for Garg's bound-based SSSP (arXiv 1812.10499).

TEST INFRASTRUCTURE ONLY.  Imported by tests/, by __graft_entry__.smoke() and
by the CPU-baseline leg of bench.py; the product library never imports it and
it never imports the product.  The arithmetic lives in oracle.c (plain,
single-threaded C); this file only marshals numpy arrays.

Parity status: see oracle.h.  Round counts of general graphs are "parity
unpinned" beyond the invariants the tests check (the paper prints none).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "_oracle.so")
_lib = None

INF = np.uint64(0xFFFFFFFFFFFFFFFF)
RULE_THR = 0
RULE_MIND = 1
LABEL_CORRECT = 2
CHEAP_FIRST = 4
ALL_UNFIXED = 8
DELTA = 16
PRED_COUNT = 32
WITNESS = 64

_STATS = ("out_scanned", "in_scanned", "active_visits", "front_visits", "reached", "max_active")

ROUND_CB = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                            ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compiles oracle.c with gcc into a shared library."""
    newest = max(os.path.getmtime(src), os.path.getmtime(_HDR))
    if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-I", _HERE, src, "-o", tmp])
        os.replace(tmp, out)
    return out


def _bind(lib):
    u32, u64, i32, vp, c_int = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32,
                                 ctypes.c_void_p, ctypes.c_int)
    lib.orc_strip_self_loops.restype = u64
    lib.orc_strip_self_loops.argtypes = [u32, vp, vp, vp]
    lib.orc_transpose.restype = c_int
    lib.orc_transpose.argtypes = [u32, vp, vp, vp, vp, vp, vp]
    lib.orc_dijkstra.restype = c_int
    lib.orc_dijkstra.argtypes = [u32, vp, vp, vp, u32, vp, vp]
    lib.orc_bellman_ford.restype = c_int
    lib.orc_bellman_ford.argtypes = [u32, vp, vp, vp, u32, vp]
    lib.orc_floyd_warshall.restype = c_int
    lib.orc_floyd_warshall.argtypes = [u32, vp, vp, vp, u32, vp]
    lib.orc_round.restype = c_int
    lib.orc_round.argtypes = [u32, vp, vp, vp, u32, u32, ctypes.c_int64, vp, vp, vp, vp, vp, vp,
                              ROUND_CB, vp]
    lib.orc_round_delta.restype = c_int
    lib.orc_round_delta.argtypes = [u32, vp, vp, vp, u32, u32, ctypes.c_int64, u64, vp, vp, vp,
                                    vp, vp, vp, ROUND_CB, vp]
    lib.orc_round_ex.restype = c_int
    lib.orc_round_ex.argtypes = [u32, vp, vp, vp, u32, u32, ctypes.c_int64, u64, u32, vp, vp, vp,
                                 vp, vp, vp, ROUND_CB, vp]
    lib.orc_prune.restype = c_int
    lib.orc_prune.argtypes = [u32, vp, vp, u32, vp]
    for f in (lib.orc_sp1, lib.orc_sp2):
        f.restype = c_int
        f.argtypes = [u32, vp, vp, vp, u32, c_int, vp, vp]
    return lib


def load(path: str | None = None):
    """Loads the oracle library (building it if needed).  A path loads another
    build of the same source (used by the mutation tests)."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _csr(g):
    """Contiguous, self-loop-free copies of a graph's CSR arrays (Sec. II)."""
    row_ptr = np.ascontiguousarray(g.row_ptr, dtype=np.uint64).copy()
    col = np.ascontiguousarray(g.col, dtype=np.uint32).copy()
    w = np.ascontiguousarray(g.w, dtype=np.uint32).copy()
    if np.any(w == 0):
        raise ValueError("edge weights must be strictly positive (Sec. I)")
    m = load().orc_strip_self_loops(g.n, row_ptr.ctypes.data, col.ctypes.data, w.ctypes.data)
    return row_ptr, col[:m].copy(), w[:m].copy()


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def dijkstra(g, s: int, lib=None):
    """Fig. 1.  Returns (dist u64[n], ops dict)."""
    lib = lib or load()
    rp, col, w = _csr(g)
    dist = np.empty(g.n, dtype=np.uint64)
    ops = np.zeros(3, dtype=np.uint64)
    _check(lib.orc_dijkstra(g.n, rp.ctypes.data, col.ctypes.data, w.ctypes.data, s,
                            dist.ctypes.data, ops.ctypes.data), "dijkstra")
    return dist, dict(inserts=int(ops[0]), adjusts=int(ops[1]), removes=int(ops[2]))


def bellman_ford(g, s: int, lib=None):
    lib = lib or load()
    rp, col, w = _csr(g)
    dist = np.empty(g.n, dtype=np.uint64)
    _check(lib.orc_bellman_ford(g.n, rp.ctypes.data, col.ctypes.data, w.ctypes.data, s,
                                dist.ctypes.data), "bellman_ford")
    return dist


def floyd_warshall(g, s: int, lib=None):
    lib = lib or load()
    rp, col, w = _csr(g)
    dist = np.empty(g.n, dtype=np.uint64)
    _check(lib.orc_floyd_warshall(g.n, rp.ctypes.data, col.ctypes.data, w.ctypes.data, s,
                                  dist.ctypes.data), "floyd_warshall")
    return dist


def transpose(g, lib=None):
    """CSC of g: (col_ptr u64[n+1], row u32[m], w_in u32[m])."""
    lib = lib or load()
    rp, col, w = _csr(g)
    m = len(col)
    col_ptr = np.empty(g.n + 1, dtype=np.uint64)
    row = np.empty(max(m, 1), dtype=np.uint32)
    w_in = np.empty(max(m, 1), dtype=np.uint32)
    _check(lib.orc_transpose(g.n, rp.ctypes.data, col.ctypes.data, w.ctypes.data,
                             col_ptr.ctypes.data, row.ctypes.data, w_in.ctypes.data), "transpose")
    return col_ptr, row[:m], w_in[:m]


@dataclass
class RoundResult:
    dist: np.ndarray         # u64[n], INF if unreachable
    parent: np.ndarray       # u32[n], 0xFFFFFFFF if unreachable
    C: np.ndarray            # u64[n] final lower bounds
    fixed_round: np.ndarray  # i32[n], -1 if never fixed
    rounds: int
    stats: dict


def round_r(g, s: int, mode: int = RULE_THR, on_round=None, lib=None,
            target: int | None = None, delta: int | None = None,
            witness_deg: int | None = None) -> RoundResult:
    """Sequential Round R (the SP_3/SP_4 round; see oracle.c).

    on_round(round, thr, minD, D, C, fixed_round) is called after every round
    with numpy views of the state (valid only during the call).  target: stop
    after the round that fixes this vertex (single-target query).  delta:
    windowed relaxation (ORC_DELTA) with this window width; None = off.
    witness_deg: stored minimum witnesses (ORC_WITNESS) for vertices of
    in-degree <= witness_deg; None = off."""
    lib = lib or load()
    rp, col, w = _csr(g)
    n = g.n
    dist = np.empty(n, dtype=np.uint64)
    parent = np.empty(n, dtype=np.uint32)
    C = np.empty(n, dtype=np.uint64)
    fr = np.empty(n, dtype=np.int32)
    rounds = ctypes.c_uint32(0)
    stats = np.zeros(len(_STATS), dtype=np.uint64)
    if on_round is not None:
        def _cb(_ctx, r, thr, minD, Dp, Cp, Fp):
            D_ = np.ctypeslib.as_array(ctypes.cast(Dp, ctypes.POINTER(ctypes.c_uint64)), (n,))
            C_ = np.ctypeslib.as_array(ctypes.cast(Cp, ctypes.POINTER(ctypes.c_uint64)), (n,))
            F_ = np.ctypeslib.as_array(ctypes.cast(Fp, ctypes.POINTER(ctypes.c_int32)), (n,))
            on_round(int(r), int(thr), int(minD), D_, C_, F_)
        cb = ROUND_CB(_cb)
    else:
        cb = ROUND_CB()
    if witness_deg is not None:
        rc = lib.orc_round_ex(n, rp.ctypes.data, col.ctypes.data, w.ctypes.data, s,
                              mode | WITNESS | (DELTA if delta is not None else 0),
                              -1 if target is None else int(target),
                              0 if delta is None else int(delta), int(witness_deg),
                              dist.ctypes.data, parent.ctypes.data, C.ctypes.data,
                              fr.ctypes.data, ctypes.byref(rounds), stats.ctypes.data, cb, None)
    elif delta is None:
        rc = lib.orc_round(n, rp.ctypes.data, col.ctypes.data, w.ctypes.data, s, mode,
                           -1 if target is None else int(target), dist.ctypes.data,
                           parent.ctypes.data, C.ctypes.data, fr.ctypes.data,
                           ctypes.byref(rounds), stats.ctypes.data, cb, None)
    else:
        rc = lib.orc_round_delta(n, rp.ctypes.data, col.ctypes.data, w.ctypes.data, s,
                                 mode | DELTA, -1 if target is None else int(target), int(delta),
                                 dist.ctypes.data, parent.ctypes.data, C.ctypes.data,
                                 fr.ctypes.data, ctypes.byref(rounds), stats.ctypes.data, cb,
                                 None)
    _check(rc, "round")
    return RoundResult(dist, parent, C, fr, int(rounds.value),
                       {k: int(v) for k, v in zip(_STATS, stats)})


def prune(g, s: int, lib=None) -> np.ndarray:
    lib = lib or load()
    rp, col, _ = _csr(g)
    removed = np.zeros(g.n, dtype=np.uint8)
    _check(lib.orc_prune(g.n, rp.ctypes.data, col.ctypes.data, s, removed.ctypes.data), "prune")
    return removed


def _sp(fn, g, s, prune_first, lib):
    rp, col, w = _csr(g)
    dist = np.empty(g.n, dtype=np.uint64)
    ops = np.zeros(4, dtype=np.uint64)
    _check(fn(g.n, rp.ctypes.data, col.ctypes.data, w.ctypes.data, s, int(prune_first),
              dist.ctypes.data, ops.ctypes.data), fn.__name__)
    return dist, dict(inserts=int(ops[0]), adjusts=int(ops[1]), removes=int(ops[2]),
                      outer=int(ops[3]))


def sp1(g, s: int, prune_first: bool = False, lib=None):
    """Fig. SP_1 (predecessor counts).  Returns (dist, heap-op counts)."""
    lib = lib or load()
    return _sp(lib.orc_sp1, g, s, prune_first, lib)


def sp2(g, s: int, prune_first: bool = False, lib=None):
    """Fig. SP_2 (predecessor counts + inWeight).  Returns (dist, heap-op counts)."""
    lib = lib or load()
    return _sp(lib.orc_sp2, g, s, prune_first, lib)
