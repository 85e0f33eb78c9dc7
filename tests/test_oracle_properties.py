"""Property-based pins of the oracle's Round R (CPU only).

Random loop-free digraphs of up to 9 vertices, with multi-edges, unreachable
parts and weights 1..20, are solved in every round mode of the oracle: the
threshold and printed minD clamps, the cheaper rules first, label-correcting
relaxation and windowed relaxation with a random window.  Each run must give
the distances of brute-force path enumeration and keep the invariants of
Lemmas 6-8 after every round (C <= cost <= D, fixed vertices at their cost,
tight parent edges).  Hypothesis is not installed everywhere; the module is
skipped where it is missing.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from tests import test_oracle_pins as pins

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

MODES = [oracle.RULE_THR, oracle.RULE_MIND, oracle.CHEAP_FIRST,
         oracle.RULE_MIND | oracle.CHEAP_FIRST, oracle.LABEL_CORRECT]


@st.composite
def small_graphs(draw):
    n = draw(st.integers(1, 9))
    m = draw(st.integers(0, 3 * n))
    edges = []
    for _ in range(m):
        u = draw(st.integers(0, n - 1))
        v = draw(st.integers(0, n - 1))
        if u != v:                                 # the oracle takes loop-free graphs
            edges.append((u, v, draw(st.integers(1, 20))))
    s = draw(st.integers(0, n - 1))
    return gg.from_edges(n, edges), s


@settings(max_examples=400, deadline=None)
@given(small_graphs(), st.sampled_from(MODES), st.one_of(st.none(), st.integers(0, 60)))
def test_round_modes_against_brute_force(gs, mode, delta):
    g, s = gs
    if mode & oracle.LABEL_CORRECT:
        delta = None                               # windowed excludes label-correcting
    cost = pins.brute_force_dist(g, s)
    r = oracle.round_r(g, s, mode=mode, delta=delta)
    assert np.array_equal(r.dist, cost)
    assert np.array_equal(oracle.dijkstra(g, s)[0], cost)
    if not mode & oracle.LABEL_CORRECT:
        # every reachable vertex ends fixed, at its cost, with C = D
        reach = cost != pins.INF
        assert np.array_equal(r.fixed_round >= 0, reach)
        assert np.array_equal(r.C[reach], cost[reach])
        pins.check_round_invariants(g, s, mode, delta=delta)


@settings(max_examples=200, deadline=None)
@given(small_graphs(), st.sampled_from([oracle.RULE_THR, oracle.RULE_MIND]))
def test_window_zero_is_label_setting(gs, mode):
    g, s = gs
    a = oracle.round_r(g, s, mode=mode)
    b = oracle.round_r(g, s, mode=mode, delta=0)
    for f in ("dist", "parent", "C", "fixed_round"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    assert a.rounds == b.rounds and a.stats == b.stats
