"""sssp_solve_noalloc, the solve for callers that cannot allocate device
memory at solve time (a framework that owns all device memory, a fixed
memory budget, a latency-critical loop that must not synchronise on
cudaMalloc): with all working state in the library's fixed scratch it must
return exactly what sssp_solve returns, call after call.

This file is named to be collected last, so a run that stops at its first
failure has already run every other test."""
import numpy as np
import pytest

import graphgen as gg

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


def test_noalloc_matches_solve_on_consecutive_calls(sssp_lib):
    torch = pytest.importorskip("torch")
    P = sssp_lib
    # Uneven out-degrees and a few hubs above the default hub degree.
    g = gg.rmat(16, 16, 1, 1000, 1810)
    wmax = int(g.w.max())
    out_off, out_adj, in_off, in_adj = device_graph(torch, g)
    h = P.sssp_create(g.n, g.row_ptr, g.col, g.w)
    try:
        cand = np.flatnonzero(g.out_degree() > 0)
        for s in (int(cand[0]), int(cand[len(cand) // 2])):
            ref, r_ref = P.sssp_solve(h, s)
            dist = torch.full((g.n,), -7, dtype=torch.int64, device="cuda")
            r = P.sssp_solve_noalloc(g.n, out_off, out_adj, in_off, in_adj, s, wmax, dist)
            torch.cuda.synchronize()
            assert r == r_ref
            assert np.array_equal(dist.cpu().numpy().view(np.uint64), ref)
    finally:
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
