"""Host logic of the autotuner: the graph-class key and the tuning cache
(read and written as JSON).  No GPU: these entry points never touch one."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

T1 = dict(hub_degree=512, chunk_edges=2048, ctas_per_sm=2, tail_items=256)
T2 = dict(hub_degree=128, chunk_edges=512, ctas_per_sm=0, tail_items=0)


@pytest.fixture()
def P():
    from paper_1812_10499_gb300 import build
    build.build()
    import paper_1812_10499_gb300 as P
    P.load()
    yield P
    P.sssp_tune_cache_open(None)          # leave an empty in-memory cache behind


def test_key_buckets(P):
    k = P.sssp_tune_key
    # R-MAT scale 22 after deduplication: 2^22 vertices, average degree ~15.6
    # (half power 8 = 2 log2(16)), hubs of 2^14..2^15, weights up to 255.
    rmat = k(1 << 22, 65_245_469, 20_000, 30_000, 255)
    assert rmat == "graph.n22.d8.o15.i15.w8.c"
    # Slightly different sizes of the same kind share the class ...
    assert k(4_000_000, 62_000_000, 17_000, 31_000, 200) == rmat
    # ... a different weight range, degree profile or size does not.
    assert k(1 << 22, 65_245_469, 20_000, 30_000, 10_000) != rmat
    assert k(1 << 22, 16 << 22, 4, 4, 255) != rmat
    assert k(1 << 20, 16 << 20, 20_000, 30_000, 255) != rmat
    # The layout bit: compact exactly when n * max weight < 2^31 - 1.
    assert k(1 << 20, 1 << 24, 8, 8, 2047).endswith(".c")
    assert k(1 << 20, 1 << 24, 8, 8, 2048).endswith(".w")
    # The grid workload: 4 neighbours, weights up to 10^4, 2^24 vertices.
    assert k(1 << 24, 67_092_480, 4, 4, 10_000) == "graph.n24.d4.o2.i2.w14.w"
    import ctypes
    assert P.load().sssp_tune_key(1, 1, 1, 1, 1, None, 96) == P.SSSP_E_INVAL
    assert P.load().sssp_tune_key(1, 1, 1, 1, 1, ctypes.create_string_buffer(95), 95) == \
        P.SSSP_E_INVAL


def test_cache_round_trip(P, tmp_path):
    path = str(tmp_path / "tune.json")
    P.sssp_tune_cache_open(path)                      # no file yet: empty
    assert P.sssp_tune_cache_get("graph.x") is None
    P.sssp_tune_cache_put("graph.x", T1)
    P.sssp_tune_cache_put("batch.y", T2)
    on_disk = json.load(open(path))                  # valid JSON, one object per key
    assert on_disk == {"graph.x": T1, "batch.y": T2}
    P.sssp_tune_cache_put("graph.x", T2)             # replaces
    P.sssp_tune_cache_open(None)                     # in-memory, empty
    assert P.sssp_tune_cache_get("graph.x") is None
    P.sssp_tune_cache_open(path)
    assert P.sssp_tune_cache_get("graph.x") == T2
    assert P.sssp_tune_cache_get("batch.y") == T2


def test_cache_rejects_bad_input(P, tmp_path):
    bad = tmp_path / "bad.json"
    for text in ('{"k": {"hub_degree": 256, "chunk_edges": 1000}}',   # chunk not a multiple of 32
                 '{"k": {"hub_degree": -1}}', '[1, 2]', '{"k": {"hub_degree": 256,'):
        bad.write_text(text)
        with pytest.raises(P.SsspError) as e:
            P.sssp_tune_cache_open(str(bad))
        assert e.value.code == P.SSSP_E_INVAL
    P.sssp_tune_cache_open(None)
    for t in (dict(T1, chunk_edges=100), dict(T1, hub_degree=0), dict(T1, ctas_per_sm=1000)):
        with pytest.raises(P.SsspError):
            P.sssp_tune_cache_put("graph.z", t)
    with pytest.raises(P.SsspError):
        P.sssp_tune_cache_put('gra"ph', T1)


def test_cache_from_the_environment(tmp_path):
    """Without an explicit open, the first use reads the file SSSP_TUNE_CACHE
    names."""
    path = tmp_path / "env.json"
    path.write_text(json.dumps({"graph.e": T1}))
    code = ("import paper_1812_10499_gb300 as P; P.load(); "
            "print(P.sssp_tune_cache_get('graph.e')['hub_degree'])")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT,
                         env={**os.environ, "SSSP_TUNE_CACHE": str(path)}, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "512"
