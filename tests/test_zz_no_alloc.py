"""sssp_solve_noalloc, the solve for callers that cannot allocate device
memory at solve time (a framework that owns all device memory, a fixed
memory budget, a latency-critical loop that must not synchronise on
cudaMalloc): with all working state in the library's fixed scratch it must
return exactly what the oracle and sssp_solve return, call after call, in
both state layouts, and whatever graph the previous call left behind.

This file is named to be collected last, so a run that stops at its first
failure has already run every other test."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def device_graph(torch, g):
    """CSR and CSC of g as CUDA tensors in the layout the entry point takes."""
    src, col, w = g.edges()
    out_off = torch.tensor(g.row_ptr.astype(np.int64), device="cuda")
    out_adj = torch.tensor(np.stack([col, w], axis=1).astype(np.int32).ravel(), device="cuda")
    order = np.argsort(col, kind="stable")
    in_cnt = np.bincount(col, minlength=g.n)
    in_off = np.zeros(g.n + 1, dtype=np.int64)
    np.cumsum(in_cnt, out=in_off[1:])
    in_adj = np.stack([src[order], w[order]], axis=1).astype(np.int32).ravel()
    return out_off, out_adj, torch.tensor(in_off, device="cuda"), torch.tensor(in_adj,
                                                                               device="cuda")


def noalloc(P, torch, g, dev, s):
    dist = torch.full((g.n,), -7, dtype=torch.int64, device="cuda")
    r = P.sssp_solve_noalloc(g.n, *dev, s, int(g.w.max()), dist)
    torch.cuda.synchronize()
    return dist.cpu().numpy().view(np.uint64), r


def check(P, torch, g, dev, h, s):
    """One no-alloc call against the oracle and against sssp_solve."""
    d, r = noalloc(P, torch, g, dev, s)
    ref = oracle.round_r(g, s)
    assert np.array_equal(d, ref.dist) and r == ref.rounds
    alone, r_alone = P.sssp_solve(h, s)
    assert np.array_equal(d, alone) and r == r_alone


def test_noalloc_matches_solve_on_consecutive_calls(sssp_lib):
    torch = pytest.importorskip("torch")
    P = sssp_lib
    # Uneven out-degrees and a few hubs above the default hub degree.
    g = gg.rmat(16, 16, 1, 1000, 1810)
    dev = device_graph(torch, g)
    h = P.sssp_create(g.n, g.row_ptr, g.col, g.w)
    try:
        assert P.sssp_layout(h) == P.SSSP_LAYOUT_COMPACT
        cand = np.flatnonzero(g.out_degree() > 0)
        for s in (int(cand[0]), int(cand[len(cand) // 2])):
            check(P, torch, g, dev, h, s)
    finally:
        P.sssp_destroy(h)


def test_noalloc_wide_records(sssp_lib):
    """Weights up to 100000 on 60000 vertices: n * max weight is above 2^31,
    so the 32-byte record layout runs (23 parent bits in the packed word)."""
    torch = pytest.importorskip("torch")
    P = sssp_lib
    g = gg.random_var_graph(60000, 2, 14, 1, 100000, 1811)
    assert g.n * int(g.w.max()) >= 1 << 31
    dev = device_graph(torch, g)
    h = P.sssp_create(g.n, g.row_ptr, g.col, g.w)
    try:
        assert P.sssp_layout(h) == P.SSSP_LAYOUT_WIDE
        for s in (0, 12345):
            check(P, torch, g, dev, h, s)
    finally:
        P.sssp_destroy(h)


def test_noalloc_scratch_reuse_across_graphs(sssp_lib):
    """A large graph, a small one, the large one again, then a wide-layout
    graph and the small one: each call clears the state it reuses, so no
    call sees what the one before left in the shared scratch."""
    torch = pytest.importorskip("torch")
    P = sssp_lib
    big = gg.rmat(17, 8, 1, 255, 1812)              # 131072 vertices: the maximum
    small = gg.random_var_graph(3000, 1, 6, 1, 50, 1813)
    wide = gg.random_var_graph(40000, 2, 10, 1, 200000, 1814)
    graphs = {"big": big, "small": small, "wide": wide}
    devs = {k: device_graph(torch, g) for k, g in graphs.items()}
    hs = {k: P.sssp_create(g.n, g.row_ptr, g.col, g.w) for k, g in graphs.items()}
    try:
        s_big = int(np.argmax(big.out_degree()))
        for k, s in (("big", s_big), ("small", 0), ("big", s_big), ("wide", 7), ("small", 0)):
            check(P, torch, graphs[k], devs[k], hs[k], s)
    finally:
        for h in hs.values():
            P.sssp_destroy(h)


def test_noalloc_rejects_graphs_beyond_its_scratch(sssp_lib):
    torch = pytest.importorskip("torch")
    P = sssp_lib
    n = 131072 + 1
    off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    dist = torch.empty(n, dtype=torch.int64, device="cuda")
    with pytest.raises(P.SsspError) as e:
        P.sssp_solve_noalloc(n, off, off, off, off, 0, 1, dist)
    assert e.value.code == -12
