"""Oracle runs of many independent queries on all host cores.

Workers are started with the "spawn" method, so they never inherit a CUDA
context, and each builds its graph from the seeded recipe (no graph is
pickled).  A job is ("batch", n, seed, i, source) for graph i of a batched
set, ("rmat", scale, seed, source) for an R-MAT graph (edge factor 16, w in
[1, 255]; kept per worker), and returns (distances, round count) of the
oracle's Round R."""
from __future__ import annotations

import multiprocessing as mp
import os

_RMAT = {}


def run(job):
    import graphgen as gg
    import oracle
    from graphgen import workloads as wl
    if job[0] == "batch":
        _, n, seed, i, s = job
        g = wl.batch_graph(n, seed, i)
    else:
        _, scale, seed, s = job
        g = _RMAT.get((scale, seed))
        if g is None:
            g = _RMAT[(scale, seed)] = gg.rmat(scale, 16, 1, 255, seed)
    r = oracle.round_r(g, s)
    return r.dist, r.rounds


def run_all(jobs, processes=None):
    """Results in job order."""
    procs = processes or min(len(jobs), os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(run, jobs, chunksize=1)
