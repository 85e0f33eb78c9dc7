"""Bit-exact parity at the benchmark's full sizes, on every workload.

The grids, the layered DAG, the 512-graph batch, the 64-source batch and the
served mix run here at exactly the sizes the benchmark times.  They are the
only runs of the 32-byte record layout with 23- and 24-bit parent fields
(n = 2^23 and 2^24) and of tens of thousands of small rounds in the cluster
tail kernel.  The weighted grid and the DAG are compared with the oracle's
Round R element by element (distances, parents, fixing rounds, final lower
bounds) plus the round count and the work counters; the unit-weight grid is
compared with its closed form; every query of the batches and of the served
mix is compared with its own oracle run (distances and rounds).
"""
import numpy as np
import pytest

import oracle
from graphgen import workloads as wl
from tests import oracle_jobs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

INF = np.uint64(0xFFFFFFFFFFFFFFFF)


def full_parity(P, g, s):
    ref = oracle.round_r(g, s)
    h = P.sssp_create(g.n, g.row_ptr, g.col, g.w)
    try:
        layout = P.sssp_layout(h)
        out = P.sssp_solve_ex(h, s, parent=True, fixed_round=True, lower=True)
    finally:
        P.sssp_destroy(h)
    for k, v in (("dist", ref.dist), ("parent", ref.parent), ("fixed_round", ref.fixed_round),
                 ("lower", ref.C)):
        assert np.array_equal(out[k], v), k
    info = out["info"]
    assert info["rounds"] == ref.rounds and info["finished"] == 1
    for k in ("out_scanned", "in_scanned", "active_visits", "front_visits", "reached"):
        assert info[k] == ref.stats[k], k
    return layout, info


def test_weighted_grid_4096(sssp_lib):
    """Grid 4096 x 4096, w in [1, 10000], source at the corner: 51,140 rounds,
    n * max weight > 2^31, so 32-byte records with 24 parent bits."""
    g, srcs = wl.grid4096()
    layout, info = full_parity(sssp_lib, g, srcs[0])
    assert layout == sssp_lib.SSSP_LAYOUT_WIDE
    assert info["rounds"] > 50000


def test_layered_dag_1024x8192(sssp_lib):
    """Layered DAG, 1024 layers of 8192 vertices, w in [1, 1000]: 32-byte
    records with 23 parent bits."""
    g, srcs = wl.dag1024()
    layout, _ = full_parity(sssp_lib, g, srcs[0])
    assert layout == sssp_lib.SSSP_LAYOUT_WIDE


def test_unit_grid_4096_closed_form(sssp_lib):
    """All weights 1 on the 4096 x 4096 grid: the round is breadth-first
    search.  Vertex (i, j) has distance i + j and is fixed in round i + j;
    its parent is the smaller of its two predecessors' ids, (i - 1, j) when
    i > 0; the loop ends after 4095 + 4095 + 1 rounds.  Every vertex is in
    the frontier once and active for one round, so the counters have closed
    forms too."""
    P = sssp_lib
    g, srcs = wl.unitgrid4096()
    R = C = 4096
    h = P.sssp_create(g.n, g.row_ptr, g.col, g.w)
    try:
        assert P.sssp_layout(h) == P.SSSP_LAYOUT_COMPACT
        out = P.sssp_solve_ex(h, srcs[0], parent=True, fixed_round=True, lower=True)
    finally:
        P.sssp_destroy(h)
    v = np.arange(g.n, dtype=np.int64)
    i, j = np.divmod(v, C)
    assert np.array_equal(out["dist"], (i + j).astype(np.uint64))
    assert np.array_equal(out["fixed_round"], (i + j).astype(np.int32))
    assert np.array_equal(out["lower"], (i + j).astype(np.uint64))
    par = np.where(i > 0, v - C, v - 1)
    par[0] = 0
    assert np.array_equal(out["parent"], par.astype(np.uint32))
    info = out["info"]
    m = 2 * (R * (C - 1) + (R - 1) * C)
    assert g.m == m
    assert info["rounds"] == (R - 1) + (C - 1) + 1 and info["finished"] == 1
    assert info["reached"] == g.n
    assert info["out_scanned"] == m
    assert info["front_visits"] == g.n
    assert info["active_visits"] == g.n - 1
    assert info["in_scanned"] == m - 2          # every in-edge but the corner's two


def test_batch_512_graphs(sssp_lib):
    """The 512 independent graphs of the batched workload (n log-uniform in
    [1K, 256K]) in one batched launch: every query equals its own oracle run
    and its own solve."""
    P = sssp_lib
    seed = wl.SEED + 3
    ns = wl.batch_sizes(512, seed)
    graphs = [wl.batch_graph(n, seed, i) for i, n in enumerate(ns)]
    srcs = [wl.batch_source(seed, i, g.n) for i, g in enumerate(graphs)]
    jobs = [("batch", n, seed, i, s) for i, (n, s) in enumerate(zip(ns, srcs))]
    refs = oracle_jobs.run_all(jobs)
    hs = [P.sssp_create(g.n, g.row_ptr, g.col, g.w) for g in graphs]
    try:
        assert max(g.n for g in graphs) > 200_000
        dists, rounds = P.sssp_solve_batch(hs, srcs)
        for i, ((rd, rr), d, r) in enumerate(zip(refs, dists, rounds)):
            assert np.array_equal(d, rd), f"query {i}"
            assert int(r) == rr, f"query {i}"
        for i in range(0, 512, 64):                  # a few against their lone solve
            alone, r_alone = P.sssp_solve(hs[i], srcs[i])
            assert np.array_equal(alone, dists[i]) and r_alone == int(rounds[i])
    finally:
        for h in hs:
            P.sssp_destroy(h)


def test_batch_64_sources_rmat18(sssp_lib):
    """64 sources on one R-MAT scale 18 graph in one batched launch."""
    P = sssp_lib
    g, srcs = wl.msrc_rmat18()
    refs = oracle_jobs.run_all([("rmat", 18, wl.SEED + 3, s) for s in srcs])
    h = P.sssp_create(g.n, g.row_ptr, g.col, g.w)
    try:
        dists, rounds = P.sssp_solve_batch([h] * len(srcs), srcs)
        for i, ((rd, rr), d, r) in enumerate(zip(refs, dists, rounds)):
            assert np.array_equal(d, rd), f"source {srcs[i]}"
            assert int(r) == rr, f"source {srcs[i]}"
    finally:
        P.sssp_destroy(h)
