"""Seeded synthetic graph generators (CSR with positive integer weights).

Shared by the tests, the oracle checks and the benchmark.  This module holds
none of the shortest-path method's arithmetic: it only builds input graphs.
The C core (graphgen.c) uses SplitMix64, so a seed gives the same graph on
every host.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "_graphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compiles graphgen.c into _graphgen.so (plain gcc, host code only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u32, u64, dbl, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
        lib.gg_random.restype = vp
        lib.gg_random.argtypes = [u32, u32, u32, u32, u64]
        lib.gg_random_var.restype = vp
        lib.gg_random_var.argtypes = [u32, u32, u32, u32, u32, u64]
        lib.gg_rmat.restype = vp
        lib.gg_rmat.argtypes = [u32, u32, dbl, dbl, dbl, u32, u32, u64]
        lib.gg_grid.restype = vp
        lib.gg_grid.argtypes = [u32, u32, u32, u32, u64]
        lib.gg_dag.restype = vp
        lib.gg_dag.argtypes = [u32, u32, u32, u32, u32, u32, u64]
        lib.gg_n.restype = u32
        lib.gg_n.argtypes = [vp]
        lib.gg_m.restype = u64
        lib.gg_m.argtypes = [vp]
        lib.gg_copy.restype = None
        lib.gg_copy.argtypes = [vp, vp, vp, vp]
        lib.gg_free.restype = None
        lib.gg_free.argtypes = [vp]
        lib.gg_uniform.restype = None
        lib.gg_uniform.argtypes = [u64, u64, u64, u64, u64, vp]
        lib.gg_unit.restype = None
        lib.gg_unit.argtypes = [u64, u64, u64, vp]
        _lib = lib
    return _lib


@dataclass
class Graph:
    """Directed graph in CSR form: out-edges of u are col/w[row_ptr[u]:row_ptr[u+1]]."""

    n: int
    row_ptr: np.ndarray  # uint64[n+1]
    col: np.ndarray      # uint32[m]
    w: np.ndarray        # uint32[m]

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1])

    def out_degree(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def edges(self):
        src = np.repeat(np.arange(self.n, dtype=np.uint32), self.out_degree().astype(np.int64))
        return src, self.col, self.w


def _take(handle) -> Graph:
    lib = _load()
    if not handle:
        raise ValueError("graph generator rejected its arguments or ran out of memory")
    try:
        n, m = lib.gg_n(handle), lib.gg_m(handle)
        row_ptr = np.empty(n + 1, dtype=np.uint64)
        col = np.empty(m, dtype=np.uint32)
        w = np.empty(m, dtype=np.uint32)
        lib.gg_copy(handle, row_ptr.ctypes.data, col.ctypes.data, w.ctypes.data)
    finally:
        lib.gg_free(handle)
    return Graph(n, row_ptr, col, w)


def random_graph(n: int, deg: int, wlo: int, whi: int, seed: int) -> Graph:
    """Each vertex gets `deg` distinct uniform non-self targets; w ~ U[wlo, whi]."""
    return _take(_load().gg_random(n, deg, wlo, whi, seed))


def random_var_graph(n: int, dmin: int, dmax: int, wlo: int, whi: int, seed: int) -> Graph:
    """Per-vertex out-degree U{dmin..dmax}, distinct uniform non-self targets."""
    return _take(_load().gg_random_var(n, dmin, dmax, wlo, whi, seed))


def rmat(scale: int, edge_factor: int, wlo: int, whi: int, seed: int,
         a: float = 0.57, b: float = 0.19, c: float = 0.19) -> Graph:
    """R-MAT, relabelled, self-loops and duplicates removed."""
    return _take(_load().gg_rmat(scale, edge_factor, a, b, c, wlo, whi, seed))


def grid(rows: int, cols: int, wlo: int, whi: int, seed: int) -> Graph:
    """4-neighbour bidirectional grid, vertex (i, j) = i * cols + j."""
    return _take(_load().gg_grid(rows, cols, wlo, whi, seed))


def dag(layers: int, width: int, deg: int, maxskip: int, wlo: int, whi: int, seed: int) -> Graph:
    """Layered DAG, edges to layer + U{1..maxskip}; edges past the last layer dropped."""
    return _take(_load().gg_dag(layers, width, deg, maxskip, wlo, whi, seed))


def out_tree(n: int, wlo: int, whi: int, seed: int) -> Graph:
    """Random out-tree rooted at 0: vertex v > 0 has one in-edge, from a
    uniform vertex with a smaller id; w ~ U[wlo, whi]."""
    v = np.arange(1, n, dtype=np.uint64)
    par = uniform(seed, 0, n, 0, 1 << 30)[1:] % v
    w = uniform(seed, 1, n, wlo, whi)[1:]
    order = np.argsort(par, kind="stable")
    row_ptr = np.zeros(n + 1, dtype=np.uint64)
    np.add.at(row_ptr, par.astype(np.int64) + 1, 1)
    return Graph(n, np.cumsum(row_ptr, dtype=np.uint64), v[order].astype(np.uint32),
                 w[order].astype(np.uint32))


def uniform(seed: int, stream: int, count: int, lo: int, hi: int) -> np.ndarray:
    out = np.empty(count, dtype=np.uint64)
    if count:
        _load().gg_uniform(seed, stream, count, lo, hi, out.ctypes.data)
    return out


def unit(seed: int, stream: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    if count:
        _load().gg_unit(seed, stream, count, out.ctypes.data)
    return out


def from_edges(n: int, edges) -> Graph:
    """CSR from a list of (src, dst, w); keeps the given order within a row."""
    edges = list(edges)
    order = sorted(range(len(edges)), key=lambda i: (edges[i][0], i))
    row_ptr = np.zeros(n + 1, dtype=np.uint64)
    for s, _, _ in edges:
        row_ptr[s + 1] += 1
    row_ptr = np.cumsum(row_ptr, dtype=np.uint64)
    col = np.array([edges[i][1] for i in order], dtype=np.uint32)
    w = np.array([edges[i][2] for i in order], dtype=np.uint32)
    return Graph(n, row_ptr, col, w)
