"""Mutation check of the oracle's pins.

Each mutant is a copy of oracle/oracle.c with one plausible mistake planted in
it (a dropped term, a wrong index, a flipped comparison, a transposed
operand).  The copy is compiled to a temporary library and run through the
same checks as test_oracle_pins.py; every mutant must fail at least one.  The
mistakes are planted on the CPU only, in temporary copies; oracle.c itself is
never modified.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.golden.fixtures import worked_example
from tests import test_oracle_pins as pins

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "oracle.c")

MUTANTS = {
    "relax adds one": ("uint64_t nd = dx + w[k];", "uint64_t nd = dx + w[k] + 1;"),
    "tie keeps larger parent": ("(nd == D[y] && x < par[y])", "(nd == D[y] && x > par[y])"),
    "threshold drops outWeight": ("thr = min_u64(thr, sat_add(D[y], outW[y]));",
                                  "thr = min_u64(thr, D[y]);"),
    "lower bound drops the clamp": ("lb = max_u64(C[x], min_u64(D[x], thr));", "lb = C[x];"),
    "in-place (Gauss-Seidel) C update": (
        "Cn[i] = max_u64(C[y], max_u64(self, best));",
        "Cn[i] = max_u64(C[y], max_u64(self, best)); C[y] = Cn[i];"),
    "self clamp ignores D": ("uint64_t self = rule_mind ? minD : min_u64(D[y], thr);",
                             "uint64_t self = rule_mind ? minD : thr;"),
    "in-edge weight of the wrong edge": ("return sat_add(lb, w_in[k]);",
                                         "return sat_add(lb, w_in[k > 0 ? k - 1 : k]);"),
    "outWeight is a max": ("mw = min_u64(mw, w[k]);", "mw = max_u64(mw, w[k]);"),
    "fix on C >= D - 1": ("int fix = (Cn[i] == D[y])", "int fix = (Cn[i] + 1 >= D[y])"),
    "dijkstra relaxes from target": ("uint64_t nd = dist[j] + w[k];",
                                     "uint64_t nd = dist[y] + w[k];"),
    "bellman-ford single sweep": ("for (uint32_t it = 0; it < n; ++it) {",
                                  "for (uint32_t it = 0; it < 1; ++it) {"),
    "floyd-warshall k innermost": (
        "for (uint32_t k = 0; k < n; ++k)\n        for (uint32_t i = 0; i < n; ++i)\n"
        "            for (uint32_t j = 0; j < n; ++j) {",
        "for (uint32_t i = 0; i < n; ++i)\n        for (uint32_t j = 0; j < n; ++j)\n"
        "            for (uint32_t k = 0; k < n; ++k) {"),
    "sp1 forgets pred decrement": ("pred[y]--;", ""),
    "transpose stores target as source": ("row[at] = u;", "row[at] = col[k];"),
    "window bound not strict": ("if (windowed && changed[y] && D[y] < window)",
                                "if (windowed && changed[y] && D[y] <= window)"),
    "window above the threshold": ("const uint64_t window = sat_add(minD, delta);",
                                   "const uint64_t window = sat_add(thr, delta);"),
    "windowed improvement not marked pending": ("if (windowed) changed[y] = 1;",
                                                "if (windowed) changed[y] = 0;"),
    "windowed frontier drops fixed vertices": ("if (windowed ? changed[y] : !label_correct)",
                                               "if (windowed ? 0 : !label_correct)"),
    "pred counts fix one relaxation early": ("(pred_count && pcnt[y] == 0)",
                                             "(pred_count && pcnt[y] <= 1)"),
    "pred counts start at the out-degree": (
        "for (uint32_t y = 0; y < n; ++y) pcnt[y] = col_ptr[y + 1] - col_ptr[y];",
        "for (uint32_t y = 0; y < n; ++y) pcnt[y] = row_ptr[y + 1] - row_ptr[y];"),
    "witness check strict": ("if (t <= wm2[y]) {", "if (t < wm2[y]) {"),
    "witness ties keep the first edge": ("(row[k] < row[kb] || (row[k] == row[kb] && w_in[k] < w_in[kb]))",
                                         "(row[k] > row[kb] || (row[k] == row[kb] && w_in[k] > w_in[kb]))"),
    "witness bound includes the minimum": ("    *m2 = second;", "    *m2 = best;"),
    "heap compares wrong way": ("if (h->key[a] != h->key[b]) return h->key[a] < h->key[b];",
                                "if (h->key[a] != h->key[b]) return h->key[a] > h->key[b];"),
}


def battery(lib):
    """The pins, run against one build of the oracle; raises on the first failure."""
    ex = worked_example()
    for name in ("A", "B", "threshold", "jacobi", "inclamp"):
        e = ex[name]
        g = gg.from_edges(e["n"], e["edges"])
        r = oracle.round_r(g, e["source"], lib=lib)
        assert r.dist.tolist() == e["dist"]
        assert r.fixed_round.tolist() == e["fixed_round"]
        assert r.parent.tolist() == e["parent"]
        assert r.rounds == e["rounds"]
        assert oracle.dijkstra(g, e["source"], lib=lib)[0].tolist() == e["dist"]
        if "sp1_inserts" in e:
            d1, o1 = oracle.sp1(g, e["source"], lib=lib)
            assert d1.tolist() == e["dist"] and o1["outer"] == e["sp1_outer"]
            assert o1["inserts"] == e["sp1_inserts"]
    for name in ("window9", "window10"):
        e = ex[name]
        g = gg.from_edges(e["n"], e["edges"])
        r = oracle.round_r(g, e["source"], lib=lib, delta=e["delta"])
        assert r.dist.tolist() == e["dist"]
        assert r.fixed_round.tolist() == e["fixed_round"]
        assert r.rounds == e["rounds"]
    for n, d, wmax, seed in pins.SMALL_CASES[::2]:
        g = pins.random_small(n, d, wmax, seed)
        ref = pins.brute_force_dist(g, 0) if n <= 8 else oracle.bellman_ford(g, 0)
        assert np.array_equal(oracle.dijkstra(g, 0, lib=lib)[0], ref)
        assert np.array_equal(oracle.floyd_warshall(g, 0, lib=lib), ref)
        assert np.array_equal(oracle.bellman_ford(g, 0, lib=lib), ref)
        pins.check_round_invariants(g, 0, lib=lib)
    g = gg.random_graph(400, 3, 1, 1, 2)
    depth = pins.bfs_depth(g, 0)
    r = oracle.round_r(g, 0, lib=lib)
    reach = depth >= 0
    assert np.array_equal(r.fixed_round[reach], depth[reach])
    assert r.rounds == int(depth.max()) + 1
    # SP_1's predecessor counts: only the scan count changes; none on a tree.
    g = gg.rmat(10, 8, 1, 255, 6)
    s = int(np.argmax(g.out_degree()))
    a = oracle.round_r(g, s, lib=lib)
    b = oracle.round_r(g, s, mode=oracle.PRED_COUNT, lib=lib)
    assert np.array_equal(a.dist, b.dist) and np.array_equal(a.C, b.C)
    assert np.array_equal(a.fixed_round, b.fixed_round) and a.rounds == b.rounds
    t = gg.out_tree(300, 1, 50, 3)
    assert oracle.round_r(t, 0, mode=oracle.PRED_COUNT, lib=lib).stats["in_scanned"] == 0
    # Stored minimum witnesses: the same state, and the scan count of an
    # independent Python count (small weights: many ties).
    for mode, (g, s) in ((oracle.RULE_THR, (gg.random_var_graph(300, 1, 12, 1, 4, 21), 0)),
                         (oracle.CHEAP_FIRST, (gg.random_var_graph(300, 1, 12, 1, 40, 22), 0))):
        a = oracle.round_r(g, s, mode=mode, lib=lib)
        b = oracle.round_r(g, s, mode=mode, witness_deg=2**32 - 1, lib=lib)
        assert np.array_equal(a.dist, b.dist) and np.array_equal(a.C, b.C)
        assert b.stats["in_scanned"] == pins.witness_scan_count(g, s, mode, 2**32 - 1)
    g = gg.random_var_graph(200, 1, 6, 1, 30, 3)
    col_ptr, row, w_in = oracle.transpose(g, lib=lib)
    fwd = sorted(pins.edges_of(g))
    bwd = sorted((int(row[k]), v, int(w_in[k]))
                 for v in range(g.n) for k in range(int(col_ptr[v]), int(col_ptr[v + 1])))
    assert fwd == bwd


def test_unmutated_oracle_passes_the_battery():
    battery(oracle.load())


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_killed(name, tmp_path):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site for {name!r} not unique"
    mutated = tmp_path / "oracle.c"
    mutated.write_text(text.replace(old, new))
    shutil.copy(os.path.join(os.path.dirname(SRC), "oracle.h"), tmp_path / "oracle.h")
    lib_path = str(tmp_path / "mutant.so")
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-I", str(tmp_path),
                           str(mutated), "-o", lib_path])
    lib = oracle.load(lib_path)
    with pytest.raises(AssertionError):
        battery(lib)
