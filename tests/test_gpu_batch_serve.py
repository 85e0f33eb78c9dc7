"""Batched and served queries give, query by query, exactly the distances and
round counts of the oracle (and of a solve on its own)."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def batch_graphs(count, seed, nmin=200, nmax=20000):
    """Independent graphs of uneven size: n log-uniform, out-degree U{4..16}."""
    u = gg.unit(seed, 1, count)
    ns = np.round(np.exp(np.log(nmin) + u * (np.log(nmax) - np.log(nmin)))).astype(int)
    graphs = [gg.random_var_graph(int(n), 4, 16, 1, 1000, seed * 1000 + i)
              for i, n in enumerate(ns)]
    srcs = [int(gg.uniform(seed, 2 + i, 1, 0, g.n - 1)[0]) for i, g in enumerate(graphs)]
    return graphs, srcs


def test_batch_independent_graphs(sssp_lib):
    P = sssp_lib
    graphs, srcs = batch_graphs(24, 3)
    hs = [P.sssp_create(g.n, g.row_ptr, g.col, g.w) for g in graphs]
    try:
        dists, rounds = P.sssp_solve_batch(hs, srcs)
        for g, s, d, r in zip(graphs, srcs, dists, rounds):
            ref = oracle.round_r(g, s)
            assert np.array_equal(d, ref.dist)
            assert int(r) == ref.rounds
        # Same again (the cached workspace is reused) and in another order.
        perm = list(reversed(range(len(hs))))
        dists2, rounds2 = P.sssp_solve_batch([hs[i] for i in perm], [srcs[i] for i in perm])
        for j, i in enumerate(perm):
            assert np.array_equal(dists2[j], dists[i]) and rounds2[j] == rounds[i]
    finally:
        for h in hs:
            P.sssp_destroy(h)


def test_batch_layouts(sssp_lib):
    """A batch runs on compact records only when every graph allows them; one
    graph with large weights switches the whole batch to wide records, and
    the same workspace then serves a compact batch again."""
    P = sssp_lib
    graphs, srcs = batch_graphs(6, 7, nmax=3000)
    big = gg.random_graph(3000, 6, 1 << 19, (1 << 20) - 1, 8)
    hs = [P.sssp_create(g.n, g.row_ptr, g.col, g.w) for g in graphs + [big]]
    try:
        assert P.sssp_layout(hs[-1]) == P.SSSP_LAYOUT_WIDE
        for sel in (list(range(6)), list(range(7)), list(range(6))):
            gs = [(graphs + [big])[i] for i in sel]
            ss = [(srcs + [0])[i] for i in sel]
            dists, rounds = P.sssp_solve_batch([hs[i] for i in sel], ss)
            for g, s, d, r in zip(gs, ss, dists, rounds):
                ref = oracle.round_r(g, s)
                assert np.array_equal(d, ref.dist) and int(r) == ref.rounds
    finally:
        for h in hs:
            P.sssp_destroy(h)


def test_batch_many_sources_one_graph(sssp_lib):
    P = sssp_lib
    g = gg.rmat(13, 16, 1, 255, 4)
    cand = np.flatnonzero(g.out_degree() > 0)
    srcs = [int(cand[int(i)]) for i in gg.uniform(4, 9, 16, 0, len(cand) - 1)]
    h = P.sssp_create(g.n, g.row_ptr, g.col, g.w)
    try:
        dists, rounds = P.sssp_solve_batch([h] * len(srcs), srcs)
        for s, d, r in zip(srcs, dists, rounds):
            ref = oracle.round_r(g, s)
            assert np.array_equal(d, ref.dist) and int(r) == ref.rounds
    finally:
        P.sssp_destroy(h)


def test_batch_with_hubs(sssp_lib):
    P = sssp_lib
    o = P.sssp_options_default()
    o.hub_degree = 8
    o.chunk_edges = 32
    graphs = [gg.rmat(11, 8, 1, 255, 20 + i) for i in range(5)]
    srcs = [int(np.argmax(g.out_degree())) for g in graphs]
    hs = [P.sssp_create(g.n, g.row_ptr, g.col, g.w, options=o) for g in graphs]
    try:
        dists, rounds = P.sssp_solve_batch(hs, srcs)
        for g, s, d, r in zip(graphs, srcs, dists, rounds):
            ref = oracle.round_r(g, s)
            assert np.array_equal(d, ref.dist) and int(r) == ref.rounds
    finally:
        for h in hs:
            P.sssp_destroy(h)


def test_batch_device(sssp_lib):
    torch = pytest.importorskip("torch")
    P = sssp_lib
    graphs, srcs = batch_graphs(6, 7)
    hs = [P.sssp_create(g.n, g.row_ptr, g.col, g.w) for g in graphs]
    try:
        outs = [torch.empty(g.n, dtype=torch.int64, device="cuda") for g in graphs]
        st = torch.cuda.Stream()
        rounds = P.sssp_solve_batch_device(hs, srcs, outs, stream=st)
        for g, s, d, r in zip(graphs, srcs, outs, rounds):
            ref = oracle.round_r(g, s)
            assert np.array_equal(d.cpu().numpy().view(np.uint64), ref.dist)
            assert int(r) == ref.rounds
    finally:
        for h in hs:
            P.sssp_destroy(h)


@pytest.mark.parametrize("manual", [False, True], ids=["thread", "manual"])
def test_serve_alone_and_in_the_mix(sssp_lib, manual):
    """Queries submitted while others run are admitted as slots free up; each
    result equals the oracle's and the query's solve on its own, and at least
    two queries shared the device in one server step.  Both with the server
    thread and with the client driving the steps."""
    P = sssp_lib
    graphs, srcs = batch_graphs(16, 11, nmin=500, nmax=30000)
    hs = [P.sssp_create(g.n, g.row_ptr, g.col, g.w) for g in graphs]
    refs = [oracle.round_r(g, s) for g, s in zip(graphs, srcs)]
    server = P.sssp_serve_open(budget_bytes=64 << 20, max_slots=4, rounds_per_step=3,
                               flags=P.SSSP_SERVE_MANUAL if manual else 0)
    try:
        outs, tickets = {}, {}
        order = [int(i) for i in np.argsort(gg.uniform(11, 50, len(hs), 0, 1 << 30))]
        done = {}
        for step, i in enumerate(order):
            outs[i] = np.zeros(graphs[i].n, dtype=np.uint64)
            tickets[i] = P.sssp_serve_submit(server, hs[i], srcs[i], outs[i])
            # poll a few outstanding tickets between submissions
            for j in list(tickets):
                if j in done:
                    continue
                st, r = P.sssp_serve_poll(server, tickets[j])
                if st == P.SSSP_OK:
                    done[j] = r
                if step % 2 == 0:
                    break
        P.sssp_serve_drain(server)
        for j in tickets:
            if j not in done:
                st, r = P.sssp_serve_poll(server, tickets[j])
                assert st == P.SSSP_OK
                done[j] = r
        stats = P.sssp_serve_stats_get(server)
        assert stats["submitted"] == stats["completed"] == len(hs)
        assert stats["queued"] == 0 and stats["inflight"] == 0
        assert stats["layout"] == P.SSSP_LAYOUT_COMPACT
        assert stats["max_inflight"] >= 2, stats        # queries overlapped on the device
        for i in range(len(hs)):
            assert np.array_equal(outs[i], refs[i].dist), f"query {i}"
            assert done[i] == refs[i].rounds
            alone, r_alone = P.sssp_solve(hs[i], srcs[i])
            assert np.array_equal(alone, outs[i]) and r_alone == done[i]
    finally:
        P.sssp_serve_close(server)
        for h in hs:
            P.sssp_destroy(h)


def test_serve_progress_without_the_client(sssp_lib):
    """The server thread runs the steps: a client that submits and then does
    nothing finds every query complete, with its timing, and the steps in
    which queries ran together."""
    import time
    P = sssp_lib
    graphs, srcs = batch_graphs(8, 12, nmin=2000, nmax=20000)
    hs = [P.sssp_create(g.n, g.row_ptr, g.col, g.w) for g in graphs]
    server = P.sssp_serve_open(budget_bytes=256 << 20, max_slots=8, rounds_per_step=4)
    try:
        outs = [np.zeros(g.n, dtype=np.uint64) for g in graphs]
        tickets = [P.sssp_serve_submit(server, h, s, o) for h, s, o in zip(hs, srcs, outs)]
        t0 = time.perf_counter()
        while P.sssp_serve_stats_get(server)["completed"] < len(hs):
            assert time.perf_counter() - t0 < 60
            time.sleep(0.05)                            # no poll, no wait, no drain
        assert P.sssp_serve_stats_get(server)["max_inflight"] >= 2
        for g, s, h, o, t in zip(graphs, srcs, hs, outs, tickets):
            ref = oracle.round_r(g, s)
            assert np.array_equal(o, ref.dist)
            st, info = P.sssp_serve_wait(server, t, 0)
            assert st == P.SSSP_OK and info["rounds"] == ref.rounds
            assert info["submit_ns"] <= info["admit_ns"] <= info["done_ns"]
            assert 1 <= info["first_step"] <= info["last_step"]
            with pytest.raises(P.SsspError) as e:      # the ticket was released
                P.sssp_serve_poll(server, t)
            assert e.value.code == P.SSSP_E_NOT_FOUND
        # wait() blocks until a later query completes
        o = np.zeros(graphs[0].n, dtype=np.uint64)
        t = P.sssp_serve_submit(server, hs[0], srcs[0], o)
        st, info = P.sssp_serve_wait(server, t, 30000)
        assert st == P.SSSP_OK and np.array_equal(o, outs[0])
    finally:
        P.sssp_serve_close(server)
        for h in hs:
            P.sssp_destroy(h)


def test_serve_wide_records(sssp_lib):
    """A graph whose distances need more than 31 bits is refused by a server
    on 16-byte records and served, bit-exactly, by one on 32-byte records
    together with ordinary graphs."""
    P = sssp_lib
    big = gg.random_graph(3000, 6, 1 << 19, (1 << 20) - 1, 8)
    graphs, srcs = batch_graphs(4, 13, nmax=5000)
    graphs.append(big)
    srcs.append(0)
    hs = [P.sssp_create(g.n, g.row_ptr, g.col, g.w) for g in graphs]
    compact = P.sssp_serve_open(budget_bytes=32 << 20, max_slots=4)
    wide = P.sssp_serve_open(budget_bytes=32 << 20, max_slots=4, flags=P.SSSP_SERVE_WIDE)
    try:
        with pytest.raises(P.SsspError) as e:
            P.sssp_serve_submit(compact, hs[-1], 0, np.zeros(big.n, dtype=np.uint64))
        assert e.value.code == P.SSSP_E_OVERFLOW
        outs = [np.zeros(g.n, dtype=np.uint64) for g in graphs]
        tickets = [P.sssp_serve_submit(wide, h, s, o) for h, s, o in zip(hs, srcs, outs)]
        P.sssp_serve_drain(wide)
        assert P.sssp_serve_stats_get(wide)["layout"] == P.SSSP_LAYOUT_WIDE
        for g, s, o, t in zip(graphs, srcs, outs, tickets):
            ref = oracle.round_r(g, s)
            st, r = P.sssp_serve_poll(wide, t)
            assert st == P.SSSP_OK and r == ref.rounds
            assert np.array_equal(o, ref.dist)
    finally:
        P.sssp_serve_close(compact)
        P.sssp_serve_close(wide)
        for h in hs:
            P.sssp_destroy(h)


def test_rule_mismatches_are_rejected(sssp_lib):
    """The server runs the default rule only; a batch needs one rule and one
    window for all its graphs.  Both refuse other handles with SSSP_E_INVAL
    before any work is queued."""
    P = sssp_lib
    g = gg.random_var_graph(300, 2, 6, 1, 50, 3)

    def make(rule=0, delta=0):
        o = P.sssp_options_default()
        o.rule = rule
        o.delta = delta
        return P.sssp_create(g.n, g.row_ptr, g.col, g.w, options=o)

    hd = make()
    hw = make(P.SSSP_RULE_WINDOWED, 40)
    hw2 = make(P.SSSP_RULE_WINDOWED, 41)
    hl = make(P.SSSP_RULE_LABEL_CORRECTING)
    server = P.sssp_serve_open(budget_bytes=16 << 20, max_slots=2)
    try:
        out = np.zeros(g.n, dtype=np.uint64)
        for h in (hw, hl):
            with pytest.raises(P.SsspError) as e:
                P.sssp_serve_submit(server, h, 0, out)
            assert e.value.code == P.SSSP_E_INVAL
        for pair in ((hw, hd), (hw, hw2), (hl, hw)):
            with pytest.raises(P.SsspError) as e:
                P.sssp_solve_batch(list(pair), [0, 0])
            assert e.value.code == P.SSSP_E_INVAL
        # the same handles alone, and a batch of one kind, still solve correctly
        d, r = P.sssp_solve_batch([hw, hw], [0, 5])
        assert np.array_equal(d[0], oracle.round_r(g, 0, delta=40).dist)
        assert int(r[1]) == oracle.round_r(g, 5, delta=40).rounds
    finally:
        P.sssp_serve_close(server)
        for h in (hd, hw, hw2, hl):
            P.sssp_destroy(h)
