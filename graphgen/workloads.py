"""The benchmark workloads as seeded recipes over the generators.

Shared by the benchmark and the full-size tests, so that both run exactly
the same inputs.  Like the generators themselves, this module holds none of
the shortest-path method's arithmetic: it only names graphs and sources.

Seeds are 1812_10499 + the workload index:
  +0  random graph n = 4096, 8 distinct out-edges, w in [1, 100], source 0
  +1  R-MAT scale 22 (edge factor 16, a/b/c/d = .57/.19/.19/.05), w in
      [1, 255], 8 sources drawn among the vertices with out-edges
  +2  grid 4096 x 4096 (w in [1, 10000] and all weights 1) and the layered
      DAG 1024 x 8192 (out-degree 8 to the next 1..4 layers, w in [1, 1000])
  +3  512 independent graphs (n log-uniform in [1K, 256K], out-degree
      U{4..16}, w in [1, 1000], one source each); 64 sources on one R-MAT
      scale 18 graph (edge factor 16, w in [1, 255])
  +4  the served query mix: graphs of the batched distribution plus R-MAT
      scale 20 graphs
"""
from __future__ import annotations

import numpy as np

from . import dag, grid, random_graph, random_var_graph, rmat, uniform, unit

SEED = 1812_10499


def random4096():
    return random_graph(4096, 8, 1, 100, SEED), [0]


def rmat_sources(g, seed, stream, count):
    """`count` sources drawn uniformly among the vertices with out-edges."""
    cand = np.flatnonzero(g.out_degree() > 0)
    return [int(cand[int(i)]) for i in uniform(seed, stream, count, 0, len(cand) - 1)]


def rmat22():
    g = rmat(22, 16, 1, 255, SEED + 1)
    return g, rmat_sources(g, SEED + 1, 7, 8)


def grid4096():
    return grid(4096, 4096, 1, 10000, SEED + 2), [0]


def unitgrid4096():
    return grid(4096, 4096, 1, 1, SEED + 2), [0]


def dag1024():
    return dag(1024, 8192, 8, 4, 1, 1000, SEED + 2), [0]


def batch_sizes(count, seed, nmin=1024, nmax=262144):
    """Vertex counts log-uniform in [nmin, nmax]."""
    u = unit(seed, 1, count)
    return [int(x) for x in np.round(np.exp(np.log(nmin) + u * (np.log(nmax) - np.log(nmin))))]


def batch_graph(n, seed, i):
    """Graph i of a batched set: out-degree U{4..16}, w in [1, 1000]."""
    return random_var_graph(n, 4, 16, 1, 1000, seed * 1000 + i)


def batch_source(seed, i, n):
    return int(uniform(seed, 2 + i, 1, 0, n - 1)[0])


def batch_graphs(count=512, seed=SEED + 3, nmin=1024, nmax=262144):
    """Independent graphs of uneven size with one seeded source each."""
    ns = batch_sizes(count, seed, nmin, nmax)
    graphs = [batch_graph(n, seed, i) for i, n in enumerate(ns)]
    return graphs, [batch_source(seed, i, g.n) for i, g in enumerate(graphs)]


def msrc_rmat18():
    """64 sources on one R-MAT scale 18 graph."""
    g = rmat(18, 16, 1, 255, SEED + 3)
    return g, rmat_sources(g, SEED + 3, 9, 64)


def serve_pool(count=48, rmat_graphs=2):
    """Graphs of the served mix: `count` of the batched distribution, then
    `rmat_graphs` R-MAT scale 20 graphs (edge factor 16, w in [1, 255])."""
    graphs, _ = batch_graphs(count, SEED + 4)
    return graphs + [rmat(20, 16, 1, 255, SEED + 4 + i) for i in range(rmat_graphs)]


def serve_queries(pool, nq, stream=3):
    """nq queries (graph index into `pool`, source): 10% on the R-MAT graphs
    (the last two of the pool), the rest spread over the others."""
    pick = unit(SEED + 4, stream, nq)
    nvar = len(pool) - 2
    which = [len(pool) - 1 - int(p * 20) % 2 if p < 0.1 else int(p * 1e6) % nvar for p in pick]
    srcs = [int(uniform(SEED + 4, 10 + i, 1, 0, pool[w].n - 1)[0]) for i, w in enumerate(which)]
    return which, srcs


def arrivals(nq, rate, stream):
    """Poisson arrival times (seconds from the start) at `rate` queries/s."""
    gaps = -np.log(1.0 - unit(SEED + 4, stream, nq)) / rate
    return np.cumsum(gaps)
