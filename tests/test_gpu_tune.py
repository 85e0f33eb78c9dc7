"""The autotuner on the GPU: any tuning leaves every result bit-identical
(distances, parents, fixing rounds, lower bounds, rounds and work counters,
checked against the oracle), the tuner's winner is set on the handle and
cached under the graph's class, new handles of that class pick it up, and
batches of graphs with different tunings stay exact."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

EXTREMES = [
    dict(hub_degree=1, chunk_edges=32, ctas_per_sm=1, tail_items=0),
    dict(hub_degree=8, chunk_edges=64, ctas_per_sm=4, tail_items=100000),
    dict(hub_degree=1024, chunk_edges=2048, ctas_per_sm=2, tail_items=16),
    dict(hub_degree=100000, chunk_edges=1 << 20, ctas_per_sm=0, tail_items=512),
]


@pytest.fixture()
def cache(sssp_lib, tmp_path):
    path = str(tmp_path / "tune.json")
    sssp_lib.sssp_tune_cache_open(path)
    yield path
    sssp_lib.sssp_tune_cache_open(None)


def full_check(P, h, g, s, ref):
    out = P.sssp_solve_ex(h, s, parent=True, fixed_round=True, lower=True)
    for k, v in (("dist", ref.dist), ("parent", ref.parent), ("fixed_round", ref.fixed_round),
                 ("lower", ref.C)):
        assert np.array_equal(out[k], v), k
    info = out["info"]
    assert info["rounds"] == ref.rounds
    for k in ("out_scanned", "in_scanned", "active_visits", "front_visits", "reached"):
        assert info[k] == ref.stats[k], k


@pytest.mark.parametrize("layout", [1, 2], ids=["wide", "compact"])
def test_any_tuning_gives_identical_results(sssp_lib, layout):
    P = sssp_lib
    g = gg.rmat(14, 16, 1, 255, 17)
    s = int(np.argmax(g.out_degree()))
    ref = oracle.round_r(g, s)
    o = P.sssp_options_default()
    o.layout = layout
    h = P.sssp_create(g.n, g.row_ptr, g.col, g.w, options=o)
    try:
        full_check(P, h, g, s, ref)
        for t in EXTREMES:
            P.sssp_set_tuning(h, t)
            assert P.sssp_get_tuning(h) == t
            full_check(P, h, g, s, ref)
        with pytest.raises(P.SsspError) as e:
            P.sssp_set_tuning(h, dict(EXTREMES[0], chunk_edges=33))
        assert e.value.code == P.SSSP_E_INVAL
    finally:
        P.sssp_destroy(h)


def test_autotune_sets_caches_and_reapplies(sssp_lib, cache):
    P = sssp_lib
    g = gg.rmat(15, 16, 1, 255, 23)
    cand = np.flatnonzero(g.out_degree() > 0)
    srcs = [int(cand[int(i)]) for i in gg.uniform(23, 1, 3, 0, len(cand) - 1)]
    refs = [oracle.round_r(g, s) for s in srcs]
    h = P.sssp_create(g.n, g.row_ptr, g.col, g.w)
    try:
        res = P.sssp_autotune(h, srcs[:2], reps=2)
        assert res["evaluated"] >= 15
        assert 0 < res["best_ms"] <= res["start_ms"] * 1.0001
        assert P.sssp_get_tuning(h) == res["best"]
        key = P.sssp_graph_key(h)
        assert P.sssp_tune_cache_get(key) == res["best"]
        for s, ref in zip(srcs, refs):
            full_check(P, h, g, s, ref)
    finally:
        P.sssp_destroy(h)
    # A new handle of the class whose options leave the choice to the library
    # starts with the cached tuning; explicit options are kept.
    h2 = P.sssp_create(g.n, g.row_ptr, g.col, g.w)
    o = P.sssp_options_default()
    o.hub_degree, o.chunk_edges = 256, 1024
    h3 = P.sssp_create(g.n, g.row_ptr, g.col, g.w, options=o)
    try:
        assert P.sssp_get_tuning(h2) == res["best"]
        assert P.sssp_get_tuning(h3)["hub_degree"] == 256
        assert P.sssp_get_tuning(h3)["chunk_edges"] == 1024
        full_check(P, h2, g, srcs[2], refs[2])
    finally:
        P.sssp_destroy(h2)
        P.sssp_destroy(h3)


def test_batch_of_graphs_with_different_tunings(sssp_lib, cache):
    """A batch runs with one tuning (the batch's cached one, else the first
    graph's) whatever the graphs' own tunings are; the batch autotuner caches
    its winner under the batch's key; every query stays exact."""
    P = sssp_lib
    graphs = [gg.rmat(12, 8, 1, 255, 40 + i) for i in range(3)]
    graphs += [gg.random_var_graph(n, 2, 12, 1, 500, 50 + n) for n in (3000, 700)]
    srcs = [int(np.argmax(g.out_degree())) for g in graphs]
    refs = [oracle.round_r(g, s) for g, s in zip(graphs, srcs)]
    hs = [P.sssp_create(g.n, g.row_ptr, g.col, g.w) for g in graphs]
    try:
        for h, t in zip(hs, EXTREMES + EXTREMES):
            P.sssp_set_tuning(h, t)
        for order in (list(range(5)), [3, 0, 4, 1, 2]):
            d, r = P.sssp_solve_batch([hs[i] for i in order], [srcs[i] for i in order])
            for j, i in enumerate(order):
                assert np.array_equal(d[j], refs[i].dist) and int(r[j]) == refs[i].rounds
        res = P.sssp_autotune_batch(hs, srcs, reps=2)
        assert P.sssp_tune_cache_get(P.sssp_batch_key(hs)) == res["best"]
        d, r = P.sssp_solve_batch(hs, srcs)
        for i in range(5):
            assert np.array_equal(d[i], refs[i].dist) and int(r[i]) == refs[i].rounds
    finally:
        for h in hs:
            P.sssp_destroy(h)
