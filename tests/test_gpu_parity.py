"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Everything here is integer work, so the bar is bit-exact equality: distances,
parents (smaller id among equal distances), the round in which every vertex
was fixed, the final lower bounds C, the round count and the work counters.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.golden.fixtures import worked_example

pytestmark = pytest.mark.gpu

INF = np.uint64(0xFFFFFFFFFFFFFFFF)
# Both per-vertex state layouts: 32-byte records and 16-byte records.
LAYOUTS = pytest.mark.parametrize("layout", [1, 2], ids=["wide", "compact"])


def make_opts(P, **kw):
    o = P.sssp_options_default()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def gpu_solve(P, g, s, max_rounds=0, **opt):
    h = P.sssp_create(g.n, g.row_ptr, g.col, g.w, options=make_opts(P, **opt) if opt else None)
    try:
        return P.sssp_solve_ex(h, s, parent=True, fixed_round=True, lower=True,
                               max_rounds=max_rounds)
    finally:
        P.sssp_destroy(h)


def assert_parity(P, g, s, mode=oracle.RULE_THR, delta=None, **opt):
    # The library's rule bits are the oracle's mode bits (minD clamp = 1,
    # label-correcting = 2, cheaper rules first = 4, windowed = 16).
    if delta is not None:
        opt.setdefault("rule", mode | P.SSSP_RULE_WINDOWED)
        opt.setdefault("delta", delta)
    elif mode != oracle.RULE_THR:
        opt.setdefault("rule", mode)
    ref = oracle.round_r(g, s, mode=mode, delta=delta)
    out = gpu_solve(P, g, s, **opt)
    assert np.array_equal(out["dist"], ref.dist)
    assert np.array_equal(out["parent"], ref.parent)
    assert np.array_equal(out["fixed_round"], ref.fixed_round)
    assert np.array_equal(out["lower"], ref.C)
    info = out["info"]
    assert info["rounds"] == ref.rounds and info["finished"] == 1
    assert info["out_scanned"] == ref.stats["out_scanned"]
    assert info["in_scanned"] == ref.stats["in_scanned"]
    assert info["active_visits"] == ref.stats["active_visits"]
    assert info["front_visits"] == ref.stats["front_visits"]
    assert info["reached"] == ref.stats["reached"]
    return out, ref


# ------------------------------------------------------------- fixtures

@LAYOUTS
@pytest.mark.parametrize("variant", ["A", "B", "threshold", "jacobi", "inclamp"])
def test_worked_examples(sssp_lib, variant, layout):
    ex = worked_example()[variant]
    g = gg.from_edges(ex["n"], ex["edges"])
    out, _ = assert_parity(sssp_lib, g, ex["source"], layout=layout)
    assert out["dist"].tolist() == ex["dist"]
    assert out["fixed_round"].tolist() == ex["fixed_round"]
    assert out["info"]["rounds"] == ex["rounds"]


@LAYOUTS
def test_random_4096_config(sssp_lib, layout):
    """Random directed graph n = 4096, 8 distinct out-edges, w in [1, 100], s = 0."""
    g = gg.random_graph(4096, 8, 1, 100, 1812_10499)
    assert_parity(sssp_lib, g, 0, layout=layout)
    assert_parity(sssp_lib, g, 0, mode=oracle.RULE_MIND, layout=layout)
    assert_parity(sssp_lib, g, 0, loop_mode=sssp_lib.SSSP_LOOP_HOST, layout=layout)
    assert_parity(sssp_lib, g, 0, loop_mode=sssp_lib.SSSP_LOOP_GRAPH, layout=layout)
    assert_parity(sssp_lib, g, 0, loop_mode=sssp_lib.SSSP_LOOP_PERSISTENT, layout=layout)


@pytest.mark.parametrize("mode", ["graph", "host"])
def test_loop_modes_rmat(sssp_lib, mode):
    """The three ways of sequencing rounds give identical results."""
    g = gg.rmat(14, 16, 1, 255, 31)
    s = int(np.argmax(g.out_degree()))
    lm = sssp_lib.SSSP_LOOP_GRAPH if mode == "graph" else sssp_lib.SSSP_LOOP_HOST
    assert_parity(sssp_lib, g, s, loop_mode=lm, hub_degree=16, chunk_edges=64)


@LAYOUTS
@pytest.mark.parametrize("seed", range(6))
def test_random_graphs_many_tiles(sssp_lib, seed, layout):
    n = [37, 300, 1000, 5000, 20000, 70001][seed]
    g = gg.random_var_graph(n, 1, 12, 1, [3, 100, 1000, 10, 255, 10000][seed], seed)
    s = int(gg.uniform(seed, 0, 1, 0, n - 1)[0])
    assert_parity(sssp_lib, g, s, layout=layout)


@LAYOUTS
@pytest.mark.parametrize("hub,chunk", [(4, 32), (8, 64), (31, 32), (32, 96)])
def test_hub_paths(sssp_lib, hub, chunk, layout):
    """Small hub thresholds push many vertices through the chunked paths."""
    g = gg.rmat(13, 8, 1, 255, hub)
    s = int(np.argmax(g.out_degree()))
    assert_parity(sssp_lib, g, s, hub_degree=hub, chunk_edges=chunk, layout=layout)
    assert_parity(sssp_lib, g, s, mode=oracle.RULE_MIND, hub_degree=hub, chunk_edges=chunk,
                  layout=layout)


@LAYOUTS
def test_degree_boundaries(sssp_lib, layout):
    """Degrees around the hub threshold (8) and chunk size (32)."""
    edges = []
    n = 400
    k = 1
    for deg in (7, 8, 9, 31, 32, 33, 64, 65, 100):
        hubv = k
        k += 1
        edges.append((0, hubv, deg))
        for j in range(deg):
            leaf = k
            k += 1
            edges.append((hubv, leaf, 1 + (j % 5)))
            edges.append((leaf, n - 1, 1 + (j % 7)))     # in-degree of n-1 grows large
    for j in range(1, k):
        edges.append((j, (j * 7) % k, 3))
    g = gg.from_edges(n, [e for e in edges if e[0] != e[1]])
    assert_parity(sssp_lib, g, 0, hub_degree=8, chunk_edges=32, layout=layout)
    assert_parity(sssp_lib, g, 0, layout=layout)


def test_star_hub_in_and_out(sssp_lib):
    """Source with 100000 out-edges; a sink with in-degree 100000."""
    n = 100_002
    leaves = np.arange(1, n - 1, dtype=np.uint32)
    w1 = (gg.uniform(1, 1, len(leaves), 1, 1000)).astype(np.uint32)
    w2 = (gg.uniform(1, 2, len(leaves), 1, 1000)).astype(np.uint32)
    src = np.concatenate([np.zeros(len(leaves), np.uint32), leaves])
    dst = np.concatenate([leaves, np.full(len(leaves), n - 1, np.uint32)])
    w = np.concatenate([w1, w2])
    order = np.lexsort((dst, src))
    row_ptr = np.zeros(n + 1, dtype=np.uint64)
    np.add.at(row_ptr, src.astype(np.int64) + 1, 1)
    g = gg.Graph(n, np.cumsum(row_ptr, dtype=np.uint64), dst[order], w[order])
    assert_parity(sssp_lib, g, 0)


def test_edge_cases(sssp_lib):
    P = sssp_lib
    # n = 1, no edges
    assert_parity(P, gg.from_edges(1, []), 0)
    # isolated vertices, source in the middle
    assert_parity(P, gg.from_edges(5, []), 2)
    # source without out-edges
    assert_parity(P, gg.from_edges(4, [(1, 2, 3), (2, 3, 1)]), 0)
    # two components
    assert_parity(P, gg.from_edges(6, [(0, 1, 2), (1, 2, 2), (3, 4, 1), (4, 5, 1), (5, 3, 1)]), 0)
    # multi-edges and self-loops (stripped, Sec. II)
    g = gg.from_edges(4, [(0, 1, 5), (0, 1, 2), (1, 1, 1), (1, 2, 4), (1, 2, 9), (2, 3, 1),
                          (3, 3, 7), (3, 0, 1)])
    out, _ = assert_parity(P, g, 0)
    assert out["dist"].tolist() == [0, 2, 6, 7]


@LAYOUTS
def test_per_round_state(sssp_lib, layout):
    """After every round r the device state equals the oracle's: D, C and the
    rounds in which vertices were fixed (the state read with max_rounds = r)."""
    g = gg.random_var_graph(700, 1, 6, 1, 50, 11)
    snaps = []
    oracle.round_r(g, 0, on_round=lambda r, thr, mD, D, C, F: snaps.append(
        (D.copy(), C.copy(), F.copy())))
    for r, (D, C, F) in enumerate(snaps, start=1):
        out = gpu_solve(sssp_lib, g, 0, max_rounds=r, layout=layout)
        assert out["info"]["rounds"] == r
        assert np.array_equal(out["dist"], D), f"D after round {r}"
        assert np.array_equal(out["lower"], C), f"C after round {r}"
        assert np.array_equal(out["fixed_round"], F), f"fixed after round {r}"


def test_unit_grid_closed_form(sssp_lib):
    """Unit weights: BFS; a 300 x 200 grid from a corner needs 498 + 1 rounds."""
    g = gg.grid(300, 200, 1, 1, 0)
    out = gpu_solve(sssp_lib, g, 0)
    i, j = np.divmod(np.arange(g.n), 200)
    assert np.array_equal(out["dist"], (i + j).astype(np.uint64))
    assert np.array_equal(out["fixed_round"], (i + j).astype(np.int32))
    assert out["info"]["rounds"] == 299 + 199 + 1


@LAYOUTS
def test_weighted_grid_and_dag(sssp_lib, layout):
    assert_parity(sssp_lib, gg.grid(200, 150, 1, 10000, 3), 0, layout=layout)
    assert_parity(sssp_lib, gg.dag(64, 512, 8, 4, 1, 1000, 2), 0, layout=layout)


@LAYOUTS
@pytest.mark.parametrize("tail_items", ["0", "64", "1000000"])
def test_cluster_tail_rounds(sssp_lib, layout, tail_items, monkeypatch):
    """Small rounds run in one thread-block cluster inside the device loop:
    never (0), from a moderate size down (64 work items), or every round
    after the first (a bound no round reaches).  Results are identical."""
    monkeypatch.setenv("SSSP_TAIL_ITEMS", tail_items)
    g = gg.rmat(14, 16, 1, 255, 17)
    s = int(np.argmax(g.out_degree()))
    assert_parity(sssp_lib, g, s, layout=layout)
    assert_parity(sssp_lib, g, s, mode=oracle.RULE_MIND, layout=layout)
    g2 = gg.random_var_graph(5000, 1, 9, 1, 300, 23)
    assert_parity(sssp_lib, g2, 7, layout=layout, hub_degree=8, chunk_edges=32)
    out, ref = assert_parity(sssp_lib, g2, 7, layout=layout)
    # Per-round state with the loop stopped early, inside the tail.
    part = gpu_solve(sssp_lib, g2, 7, max_rounds=ref.rounds - 3, layout=layout)
    assert part["info"]["rounds"] == ref.rounds - 3


@LAYOUTS
@pytest.mark.parametrize("loop", ["graph", "host", "persistent"])
def test_single_target_query(sssp_lib, layout, loop):
    """Stopping at the round that fixes the target: the whole state (D,
    parents, C, fixing rounds, counters) equals the oracle's single-target
    run, and sssp_solve_to returns the target's distance."""
    P = sssp_lib
    lm = {"graph": P.SSSP_LOOP_GRAPH, "host": P.SSSP_LOOP_HOST,
          "persistent": P.SSSP_LOOP_PERSISTENT}[loop]
    g = gg.random_var_graph(3000, 0, 8, 1, 200, 43)
    full = oracle.round_r(g, 0)
    reach = np.flatnonzero(full.fixed_round >= 0)
    unreach = np.flatnonzero(full.fixed_round < 0)
    assert len(unreach) > 0
    order = reach[np.argsort(full.fixed_round[reach], kind="stable")]
    targets = [0, int(order[1]), int(order[len(order) // 2]), int(order[-1]), int(unreach[0])]
    h = P.sssp_create(g.n, g.row_ptr, g.col, g.w, options=make_opts(P, layout=layout, loop_mode=lm))
    try:
        for t in targets:
            ref = oracle.round_r(g, 0, target=t)
            out = P.sssp_solve_ex(h, 0, parent=True, fixed_round=True, lower=True, target=t)
            assert np.array_equal(out["dist"], ref.dist), t
            assert np.array_equal(out["parent"], ref.parent), t
            assert np.array_equal(out["fixed_round"], ref.fixed_round), t
            assert np.array_equal(out["lower"], ref.C), t
            info = out["info"]
            assert info["rounds"] == ref.rounds
            assert info["finished"] == (1 if full.fixed_round[t] < 0 else 0)
            assert info["out_scanned"] == ref.stats["out_scanned"]
            assert info["in_scanned"] == ref.stats["in_scanned"]
            d, r = P.sssp_solve_to(h, 0, t)
            assert d == int(full.dist[t]) and r == ref.rounds
        with pytest.raises(P.SsspError) as e:
            P.sssp_solve_to(h, 0, g.n)
        assert e.value.code == -3
    finally:
        P.sssp_destroy(h)


LC_MODES = pytest.mark.parametrize("mode", [oracle.LABEL_CORRECT,
                                            oracle.LABEL_CORRECT | oracle.RULE_MIND],
                                   ids=["lc", "lc-mind"])


@LAYOUTS
@LC_MODES
@pytest.mark.parametrize("loop", ["graph", "host", "persistent"])
def test_label_correcting(sssp_lib, layout, mode, loop):
    """SP_4 step 3 as printed: every vertex whose D changed is relaxed again
    the next round.  Bit-exact with the oracle's label-correcting Round R on
    random, skewed (with small hub thresholds) and grid graphs."""
    P = sssp_lib
    lm = {"graph": P.SSSP_LOOP_GRAPH, "host": P.SSSP_LOOP_HOST,
          "persistent": P.SSSP_LOOP_PERSISTENT}[loop]
    g = gg.random_graph(4096, 8, 1, 100, 1812_10499)
    assert_parity(P, g, 0, mode=mode, layout=layout, loop_mode=lm)
    g = gg.rmat(13, 8, 1, 255, 5)
    s = int(np.argmax(g.out_degree()))
    assert_parity(P, g, s, mode=mode, layout=layout, loop_mode=lm)
    assert_parity(P, g, s, mode=mode, layout=layout, loop_mode=lm, hub_degree=8, chunk_edges=32)
    assert_parity(P, gg.grid(60, 50, 1, 1000, 3), 0, mode=mode, layout=layout, loop_mode=lm)
    g = gg.random_var_graph(2000, 0, 7, 1, 50, 9)                     # some unreachable
    assert_parity(P, g, 3, mode=mode, layout=layout, loop_mode=lm)


@LC_MODES
def test_label_correcting_per_round_state(sssp_lib, mode, monkeypatch):
    """The state after every round equals the oracle's (solves stopped with
    max_rounds), with the small rounds in the cluster tail kernel too."""
    monkeypatch.setenv("SSSP_TAIL_ITEMS", "1000000")
    g = gg.random_var_graph(700, 1, 6, 1, 50, 12)
    snaps = []
    ref = oracle.round_r(g, 0, mode=mode, on_round=lambda r, thr, mD, D, C, F: snaps.append(
        (D.copy(), C.copy(), F.copy())))
    assert ref.rounds == len(snaps)
    for r, (D, C, F) in enumerate(snaps, start=1):
        out = gpu_solve(sssp_lib, g, 0, max_rounds=r, rule=mode)
        assert out["info"]["rounds"] == r
        assert np.array_equal(out["dist"], D), f"D after round {r}"
        assert np.array_equal(out["lower"], C), f"C after round {r}"
        assert np.array_equal(out["fixed_round"], F), f"fixed after round {r}"


def test_label_correcting_batch(sssp_lib):
    P = sssp_lib
    o = P.sssp_options_default()
    o.rule = P.SSSP_RULE_LABEL_CORRECTING
    graphs = [gg.random_var_graph(n, 2, 10, 1, 500, 60 + i) for i, n in enumerate((300, 5000, 1200, 64))]
    hs = [P.sssp_create(g.n, g.row_ptr, g.col, g.w, options=o) for g in graphs]
    try:
        srcs = [0, 7, 100, 5]
        dists, rounds = P.sssp_solve_batch(hs, srcs)
        for g, s, d, r in zip(graphs, srcs, dists, rounds):
            ref = oracle.round_r(g, s, mode=oracle.LABEL_CORRECT)
            assert np.array_equal(d, ref.dist) and int(r) == ref.rounds
    finally:
        for h in hs:
            P.sssp_destroy(h)


@LAYOUTS
@pytest.mark.parametrize("loop", ["graph", "host", "persistent"])
@pytest.mark.parametrize("delta", [0, 3, 40, 2**64 - 1], ids=["d0", "d3", "d40", "dinf"])
def test_windowed(sssp_lib, layout, loop, delta):
    """Windowed relaxation (the lower bounds with a Delta-stepping window):
    bit-exact with the oracle -- state, round count and counters -- on
    random, skewed (small hub thresholds too), grid, layered and partly
    unreachable graphs, from the label-setting end (delta 0) to the
    label-correcting end."""
    P = sssp_lib
    lm = {"graph": P.SSSP_LOOP_GRAPH, "host": P.SSSP_LOOP_HOST,
          "persistent": P.SSSP_LOOP_PERSISTENT}[loop]
    kw = dict(delta=delta, layout=layout, loop_mode=lm)
    assert_parity(P, gg.random_graph(4096, 8, 1, 100, 1812_10499), 0, **kw)
    g = gg.rmat(13, 8, 1, 255, 5)
    s = int(np.argmax(g.out_degree()))
    assert_parity(P, g, s, **kw)
    assert_parity(P, g, s, hub_degree=8, chunk_edges=32, **kw)
    assert_parity(P, gg.grid(60, 50, 1, 1000, 3), 0, **kw)
    assert_parity(P, gg.dag(10, 200, 6, 3, 1, 300, 4), 0, **kw)
    assert_parity(P, gg.random_var_graph(2000, 0, 7, 1, 50, 9), 3, **kw)


@LAYOUTS
def test_windowed_single_target(sssp_lib, layout):
    """Windowed relaxation stopped at the round that fixes a target: the
    state and counters equal the oracle's windowed single-target run."""
    P = sssp_lib
    g = gg.random_var_graph(3000, 0, 8, 1, 200, 43)
    delta = 60
    full = oracle.round_r(g, 0, delta=delta)
    reach = np.flatnonzero(full.fixed_round >= 0)
    unreach = np.flatnonzero(full.fixed_round < 0)
    order = reach[np.argsort(full.fixed_round[reach], kind="stable")]
    targets = [0, int(order[1]), int(order[len(order) // 2]), int(order[-1]), int(unreach[0])]
    h = P.sssp_create(g.n, g.row_ptr, g.col, g.w,
                      options=make_opts(P, layout=layout, rule=P.SSSP_RULE_WINDOWED, delta=delta))
    try:
        for t in targets:
            ref = oracle.round_r(g, 0, target=t, delta=delta)
            out = P.sssp_solve_ex(h, 0, parent=True, fixed_round=True, lower=True, target=t)
            for k, v in (("dist", ref.dist), ("parent", ref.parent),
                         ("fixed_round", ref.fixed_round), ("lower", ref.C)):
                assert np.array_equal(out[k], v), (t, k)
            info = out["info"]
            assert info["rounds"] == ref.rounds
            # a run that reaches the end of the loop counts as finished
            assert info["finished"] == (1 if ref.rounds == full.rounds else 0)
            for k in ("out_scanned", "in_scanned", "active_visits", "front_visits"):
                assert info[k] == ref.stats[k], (t, k)
    finally:
        P.sssp_destroy(h)


@LAYOUTS
@pytest.mark.parametrize("variant", ["window9", "window10"])
def test_windowed_hand_derived_trace(sssp_lib, layout, variant):
    ex = worked_example()[variant]
    g = gg.from_edges(ex["n"], ex["edges"])
    out, _ = assert_parity(sssp_lib, g, ex["source"], delta=ex["delta"], layout=layout)
    assert out["info"]["rounds"] == ex["rounds"]
    assert out["fixed_round"].tolist() == ex["fixed_round"]


@pytest.mark.parametrize("base", [oracle.RULE_THR, oracle.RULE_MIND, oracle.CHEAP_FIRST],
                         ids=["thr", "mind", "cheap"])
@pytest.mark.parametrize("tail", ["cluster", "grid"])
def test_windowed_per_round_state(sssp_lib, base, tail, monkeypatch):
    """The state after every round equals the oracle's (solves stopped with
    max_rounds), with every round in the cluster tail kernel or none."""
    monkeypatch.setenv("SSSP_TAIL_ITEMS", "1000000" if tail == "cluster" else "0")
    g = gg.random_var_graph(700, 1, 6, 1, 50, 12)
    for delta in (5, 60):
        snaps = []
        ref = oracle.round_r(g, 0, mode=base, delta=delta,
                             on_round=lambda r, thr, mD, D, C, F: snaps.append(
                                 (D.copy(), C.copy(), F.copy())))
        assert ref.rounds == len(snaps)
        for r, (D, C, F) in enumerate(snaps, start=1):
            out = gpu_solve(sssp_lib, g, 0, max_rounds=r, rule=base | sssp_lib.SSSP_RULE_WINDOWED,
                            delta=delta)
            assert out["info"]["rounds"] == r
            assert np.array_equal(out["dist"], D), f"D after round {r}"
            assert np.array_equal(out["lower"], C), f"C after round {r}"
            assert np.array_equal(out["fixed_round"], F), f"fixed after round {r}"


def test_windowed_batch(sssp_lib):
    """Several graphs in one batched launch, windowed: each equals its own
    oracle run (distances and round count)."""
    P = sssp_lib
    o = P.sssp_options_default()
    o.rule = P.SSSP_RULE_WINDOWED
    o.delta = 120
    graphs = [gg.random_var_graph(n, 2, 10, 1, 500, 70 + i) for i, n in enumerate((300, 5000, 1200, 64))]
    graphs.append(gg.grid(40, 30, 1, 1000, 75))
    hs = [P.sssp_create(g.n, g.row_ptr, g.col, g.w, options=o) for g in graphs]
    try:
        srcs = [0, 7, 100, 5, 0]
        dists, rounds = P.sssp_solve_batch(hs, srcs)
        for g, s, d, r in zip(graphs, srcs, dists, rounds):
            ref = oracle.round_r(g, s, delta=120)
            assert np.array_equal(d, ref.dist) and int(r) == ref.rounds
    finally:
        for h in hs:
            P.sssp_destroy(h)


@LAYOUTS
@pytest.mark.parametrize("base", [oracle.RULE_THR, oracle.RULE_MIND, oracle.LABEL_CORRECT],
                         ids=["thr", "mind", "lc"])
def test_cheap_rules_first(sssp_lib, layout, base):
    """Cheaper fixing rules before the in-edge scan: bit-exact with the
    oracle in the same mode, counters included (fewer in-edges read)."""
    P = sssp_lib
    mode = base | oracle.CHEAP_FIRST
    assert_parity(P, gg.random_graph(4096, 8, 1, 100, 1812_10499), 0, mode=mode, layout=layout)
    g = gg.rmat(13, 8, 1, 255, 6)
    s = int(np.argmax(g.out_degree()))
    assert_parity(P, g, s, mode=mode, layout=layout)
    assert_parity(P, g, s, mode=mode, layout=layout, hub_degree=8, chunk_edges=32)
    assert_parity(P, gg.grid(50, 40, 1, 100, 2), 0, mode=mode, layout=layout,
                  loop_mode=P.SSSP_LOOP_PERSISTENT)


@LAYOUTS
@pytest.mark.parametrize("base", [oracle.RULE_THR, oracle.RULE_MIND, oracle.CHEAP_FIRST],
                         ids=["thr", "mind", "cheap"])
def test_pred_counts(sssp_lib, layout, base):
    """SP_1's predecessor counts: bit-exact with the oracle in the same mode,
    counters included (fewer in-edges read), through the hub paths and every
    loop mode."""
    P = sssp_lib
    mode = base | oracle.PRED_COUNT
    assert_parity(P, gg.random_graph(4096, 8, 1, 100, 1812_10499), 0, mode=mode, layout=layout)
    g = gg.rmat(13, 8, 1, 255, 6)
    s = int(np.argmax(g.out_degree()))
    assert_parity(P, g, s, mode=mode, layout=layout)
    assert_parity(P, g, s, mode=mode, layout=layout, hub_degree=8, chunk_edges=32)
    assert_parity(P, g, s, mode=mode, layout=layout, loop_mode=P.SSSP_LOOP_HOST)
    assert_parity(P, gg.grid(50, 40, 1, 100, 2), 0, mode=mode, layout=layout,
                  loop_mode=P.SSSP_LOOP_PERSISTENT)
    assert_parity(P, gg.dag(20, 64, 5, 3, 1, 100, 7), 0, mode=mode, layout=layout)


@pytest.mark.parametrize("tail", ["cluster", "grid"])
def test_pred_counts_per_round_state(sssp_lib, tail, monkeypatch):
    """The state after every round equals the oracle's (solves stopped with
    max_rounds), with every round in the cluster tail kernel or none."""
    monkeypatch.setenv("SSSP_TAIL_ITEMS", "1000000" if tail == "cluster" else "0")
    g = gg.random_var_graph(700, 1, 6, 1, 50, 12)
    mode = oracle.CHEAP_FIRST | oracle.PRED_COUNT
    snaps = []
    ref = oracle.round_r(g, 0, mode=mode, on_round=lambda r, thr, mD, D, C, F: snaps.append(
        (D.copy(), C.copy(), F.copy())))
    assert ref.rounds == len(snaps)
    for r, (D, C, F) in enumerate(snaps, start=1):
        out = gpu_solve(sssp_lib, g, 0, max_rounds=r, rule=mode)
        assert out["info"]["rounds"] == r
        assert np.array_equal(out["dist"], D), f"D after round {r}"
        assert np.array_equal(out["lower"], C), f"C after round {r}"
        assert np.array_equal(out["fixed_round"], F), f"fixed after round {r}"


@LAYOUTS
def test_pred_counts_on_an_out_tree(sssp_lib, layout):
    """On an out-tree every discovered vertex's one in-neighbour is fixed and
    has relaxed it: no in-edge is read, and the distances are Dijkstra's."""
    P = sssp_lib
    g = gg.out_tree(20000, 1, 50, 5)
    out, ref = assert_parity(P, g, 0, mode=oracle.PRED_COUNT, layout=layout)
    assert out["info"]["in_scanned"] == 0
    assert out["info"]["reached"] == g.n


def test_pred_counts_batch(sssp_lib):
    """Several graphs in one batched launch with predecessor counts: each
    equals its own oracle run (distances and round count)."""
    P = sssp_lib
    o = P.sssp_options_default()
    o.rule = P.SSSP_RULE_PRED_COUNT | P.SSSP_RULE_CHEAP_FIRST
    graphs = [gg.random_var_graph(n, 2, 10, 1, 500, 80 + i) for i, n in enumerate((300, 5000, 1200, 64))]
    graphs += [gg.grid(40, 30, 1, 1000, 85), gg.out_tree(3000, 1, 500, 86)]
    hs = [P.sssp_create(g.n, g.row_ptr, g.col, g.w, options=o) for g in graphs]
    try:
        srcs = [0, 7, 100, 5, 0, 0]
        dists, rounds = P.sssp_solve_batch(hs, srcs)
        for g, s, d, r in zip(graphs, srcs, dists, rounds):
            ref = oracle.round_r(g, s, mode=oracle.PRED_COUNT | oracle.CHEAP_FIRST)
            assert np.array_equal(d, ref.dist) and int(r) == ref.rounds
    finally:
        for h in hs:
            P.sssp_destroy(h)


@pytest.mark.parametrize("slot", [0, 7, 15])
def test_control_block_slot(sssp_lib, slot, monkeypatch):
    """The control block's placement (chosen by a latency probe among 16
    slots, here forced) changes no result: single queries in every loop mode
    and a batch whose per-query scalars do not fit beside it."""
    monkeypatch.setenv("SSSP_HOT_SLOT", str(slot))
    P = sssp_lib
    g = gg.random_var_graph(3000, 1, 8, 1, 200, 41)
    for lm in (P.SSSP_LOOP_GRAPH, P.SSSP_LOOP_HOST, P.SSSP_LOOP_PERSISTENT):
        assert_parity(P, g, 0, loop_mode=lm)
    graphs = [gg.random_var_graph(200 + 7 * i, 1, 6, 1, 50, 90 + i) for i in range(64)]
    hs = [P.sssp_create(x.n, x.row_ptr, x.col, x.w) for x in graphs]
    try:
        dists, rounds = P.sssp_solve_batch(hs, [0] * len(graphs))
        for x, d, r in zip(graphs, dists, rounds):
            ref = oracle.round_r(x, 0)
            assert np.array_equal(d, ref.dist) and int(r) == ref.rounds
    finally:
        for h in hs:
            P.sssp_destroy(h)


def test_kernel_launch_count(sssp_lib, monkeypatch):
    """The solve reports the kernels it launched: four start/output kernels
    plus the round kernels of its loop mode."""
    P = sssp_lib
    g = gg.random_var_graph(3000, 1, 8, 1, 200, 41)
    ref = oracle.round_r(g, 0)
    r = ref.rounds
    host = gpu_solve(P, g, 0, loop_mode=P.SSSP_LOOP_HOST)["info"]
    assert host["kernel_launches"] == 4 + 2 * 16 * ((r + 15) // 16)   # groups of 16 rounds
    pers = gpu_solve(P, g, 0, loop_mode=P.SSSP_LOOP_PERSISTENT)["info"]
    assert pers["kernel_launches"] == 5
    monkeypatch.setenv("SSSP_TAIL_ITEMS", "0")
    plain = gpu_solve(P, g, 0)["info"]
    assert plain["kernel_launches"] == 4 + 2 * r                       # relax + cupdate per round
    monkeypatch.setenv("SSSP_TAIL_ITEMS", "1000000")
    tail = gpu_solve(P, g, 0)["info"]                                  # rounds 2.. in the cluster
    assert 4 + 3 <= tail["kernel_launches"] <= 4 + 3 * 2


def test_device_wait_limit_without_a_fault(sssp_lib):
    """Failure detection on the GPU without a fault: the persistent kernel's
    grid barrier is run with one CTA that never arrives; the others give up
    after the limit, flag it and exit; the host reads SSSP_E_DEVICE_TIMEOUT
    and the context keeps working."""
    import time
    P = sssp_lib
    t0 = time.perf_counter()
    rc = P.sssp_selftest_barrier_timeout(200)
    dt = time.perf_counter() - t0
    assert rc == -6
    assert 0.15 < dt < 10.0
    assert_parity(P, gg.random_graph(4096, 8, 1, 100, 1812_10499), 0,
                  loop_mode=P.SSSP_LOOP_PERSISTENT)


def test_layout_selection(sssp_lib):
    """The automatic layout is compact exactly when n * max weight < 2^31 - 1;
    a graph whose distances need more than 31 bits solves with wide records,
    and asking for compact records there is refused."""
    P = sssp_lib
    small = gg.random_graph(4096, 8, 1, 100, 5)
    big = gg.random_graph(4096, 8, 1 << 19, (1 << 20) - 1, 5)     # 4096 * 2^20 = 2^32
    for g, want in ((small, P.SSSP_LAYOUT_COMPACT), (big, P.SSSP_LAYOUT_WIDE)):
        h = P.sssp_create(g.n, g.row_ptr, g.col, g.w)
        try:
            assert P.sssp_layout(h) == want
        finally:
            P.sssp_destroy(h)
    out, ref = assert_parity(P, big, 0)
    assert int(ref.dist[ref.dist != INF].max()) >= 1 << 21
    with pytest.raises(P.SsspError) as e:
        P.sssp_create(big.n, big.row_ptr, big.col, big.w,
                      options=make_opts(P, layout=P.SSSP_LAYOUT_COMPACT))
    assert e.value.code == -4


def test_solve_and_solve_device(sssp_lib):
    torch = pytest.importorskip("torch")
    P = sssp_lib
    g = gg.rmat(14, 16, 1, 255, 9)
    s = int(np.argmax(g.out_degree()))
    ref = oracle.round_r(g, s)
    h = P.sssp_create(g.n, g.row_ptr, g.col, g.w)
    try:
        d, r = P.sssp_solve(h, s)
        assert np.array_equal(d, ref.dist) and r == ref.rounds
        st = torch.cuda.Stream()
        dd = torch.empty(g.n, dtype=torch.int64, device="cuda")
        with torch.cuda.stream(st):
            P.sssp_solve_device(h, s, dd, stream=st)
        st.synchronize()
        assert np.array_equal(dd.cpu().numpy().view(np.uint64), ref.dist)
        assert P.sssp_solve_device(h, s, dd, stream=st, want_rounds=True) == ref.rounds
    finally:
        P.sssp_destroy(h)


def test_host_outputs_and_reused_output_array(sssp_lib):
    """Host outputs of sssp_solve_ex, and sssp_solve writing into a caller's
    reused array, equal the oracle's on consecutive calls."""
    P = sssp_lib
    g = gg.rmat(13, 16, 1, 255, 21)
    s = int(np.argmax(g.out_degree()))
    ref = oracle.round_r(g, s)
    h = P.sssp_create(g.n, g.row_ptr, g.col, g.w)
    out_arr = np.full(g.n, 7, dtype=np.uint64)
    try:
        for _ in range(2):
            out = P.sssp_solve_ex(h, s, parent=True, fixed_round=True, lower=True)
            assert np.array_equal(out["dist"], ref.dist)
            assert np.array_equal(out["parent"], ref.parent)
            assert np.array_equal(out["fixed_round"], ref.fixed_round)
            assert np.array_equal(out["lower"], ref.C)
            d, r = P.sssp_solve(h, s, out=out_arr)
            assert d is out_arr
            assert np.array_equal(d, ref.dist) and r == ref.rounds
        with pytest.raises(P.SsspError):
            P.sssp_solve(h, s, out=np.zeros(g.n, dtype=np.int32))
    finally:
        P.sssp_destroy(h)


def test_page_locked_output_array(sssp_lib):
    """host_empty gives a page-locked array; solves into it (reused across
    calls) equal solves into a pageable one."""
    P = sssp_lib
    g = gg.rmat(12, 8, 1, 255, 31)
    h = P.sssp_create(g.n, g.row_ptr, g.col, g.w)
    try:
        pinned = P.host_empty(g.n)
        assert pinned.dtype == np.uint64 and pinned.shape == (g.n,)
        for s in (0, 5, 77):
            ref = oracle.round_r(g, s).dist
            d1, _ = P.sssp_solve(h, s, out=pinned)
            assert d1 is pinned
            assert np.array_equal(pinned, ref)
            assert np.array_equal(P.sssp_solve(h, s, out=np.empty(g.n, np.uint64))[0], ref)
        del pinned, d1
    finally:
        P.sssp_destroy(h)


def test_given_csc_and_torch_allocator(sssp_lib):
    torch = pytest.importorskip("torch")
    P = sssp_lib
    g = gg.random_var_graph(3000, 2, 9, 1, 77, 5)
    col_ptr, row, w_in = oracle.transpose(g)
    ref = oracle.round_r(g, 3)
    before = torch.cuda.memory_allocated()
    opt = P.torch_allocator_options()
    h = P.sssp_create(g.n, g.row_ptr, g.col, g.w, col_ptr, row, w_in, options=opt)
    try:
        assert torch.cuda.memory_allocated() > before   # device memory came from torch
        out = P.sssp_solve_ex(h, 3, fixed_round=True)
        assert np.array_equal(out["dist"], ref.dist)
        assert np.array_equal(out["fixed_round"], ref.fixed_round)
    finally:
        P.sssp_destroy(h)


def test_source_range(sssp_lib):
    P = sssp_lib
    g = gg.random_graph(16, 2, 1, 5, 1)
    h = P.sssp_create(g.n, g.row_ptr, g.col, g.w)
    try:
        with pytest.raises(P.SsspError) as e:
            P.sssp_solve(h, 16)
        assert e.value.code == -3
    finally:
        P.sssp_destroy(h)


@pytest.mark.slow
def test_rmat22_full_size(sssp_lib):
    """R-MAT scale 22, edge factor 16, w in [1, 255], one source of the
    benchmark's eight: bit-exact distances, fixing rounds and counters."""
    g = gg.rmat(22, 16, 1, 255, 1812_10499 + 1)
    outdeg = g.out_degree()
    cand = np.flatnonzero(outdeg > 0)
    s = int(cand[int(gg.uniform(1812_10499 + 1, 7, 1, 0, len(cand) - 1)[0])])
    assert_parity(sssp_lib, g, s)


@pytest.mark.parametrize("loop", ["graph", "host", "persistent"])
def test_profiled_solve_splits_the_work_by_kernel(sssp_lib, loop):
    """A profiled solve launches the round kernels from the host in the loop
    mode's own schedule (the device loop: k_relax, k_cupdate, then the
    cluster tail kernel): its results are bit-exact, and the work counters
    it attributes to the kernels add up to the solve's counters."""
    P = sssp_lib
    lm = {"graph": P.SSSP_LOOP_GRAPH, "host": P.SSSP_LOOP_HOST,
          "persistent": P.SSSP_LOOP_PERSISTENT}[loop]
    g = gg.rmat(14, 16, 1, 255, 17)
    s = int(np.argmax(g.out_degree()))
    ref = oracle.round_r(g, s)
    h = P.sssp_create(g.n, g.row_ptr, g.col, g.w, options=make_opts(P, loop_mode=lm))
    try:
        P.sssp_profile(h, True)
        out = P.sssp_solve_ex(h, s, parent=True, fixed_round=True, lower=True)
        prof = P.sssp_profile(h, False)
        relax, cup, tail, tail_rounds, ctr = P.sssp_profile_rounds(h)
    finally:
        P.sssp_destroy(h)
    for k, v in (("dist", ref.dist), ("parent", ref.parent), ("fixed_round", ref.fixed_round),
                 ("lower", ref.C)):
        assert np.array_equal(out[k], v), k
    info = out["info"]
    assert info["rounds"] == ref.rounds
    for k in ("out_scanned", "in_scanned", "active_visits", "front_visits"):
        assert prof["grid_counters"][k] + prof["tail_counters"][k] == info[k] == ref.stats[k], k
    n_it = len(cup)
    assert prof["cupdate_launches"] == prof["relax_launches"] == n_it
    if loop == "graph":
        # every iteration's k_cupdate closes one round, k_tail the rounds after it
        assert prof["tail_launches"] == n_it and int(tail_rounds.sum()) == prof["tail_rounds"]
        assert n_it + prof["tail_rounds"] == ref.rounds
        assert prof["tail_rounds"] > 0 and prof["tail_counters"]["in_scanned"] > 0
        assert info["kernel_launches"] == 4 + 3 * n_it
        # per-iteration counters add up to the grid kernels' totals
        for j, k in enumerate(("out_scanned", "in_scanned", "active_visits", "front_visits")):
            assert int(ctr[:, j].sum()) == prof["grid_counters"][k]
    else:
        assert n_it == ref.rounds and prof["tail_launches"] == 0
        assert prof["tail_counters"] == {k: 0 for k in prof["tail_counters"]}
