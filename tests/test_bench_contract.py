"""The benchmark's contract on the host: the reference arm (the oracle, no
GPU) prints one JSON line with the keys the driver reads, and the traffic
figure of a committed ncu summary is withheld once the kernels' sources no
longer match the ones it was captured from."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--config", "random4096", "--steps", "3", "--warmup", "1"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "GTEPS" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["vs_baseline"] is None


def test_traffic_withheld_when_the_kernels_changed(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    sha = bench.kernel_source_sha256()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps({
        "k_cupdate/x": {"kernel_source_sha256": sha, "traffic_bytes_per_launch": 123,
                        "how": "ncu"},
        "k_relax/x": {"kernel_source_sha256": "00", "traffic_bytes_per_launch": 456},
        "k_tail/x": {"kernel_source_sha256": sha, "dram_per_algorithmic_byte": 1.25}}))
    (tmp_path / "paper_1812_10499_gb300").symlink_to(os.path.join(ROOT, "paper_1812_10499_gb300"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("k_cupdate", "x")[0] == 123.0
    t, why = bench.measured_traffic("k_relax", "x")
    assert t is None and "stale" in why
    assert bench.measured_traffic("k_cupdate", "missing") == (None, None)
    # a ratio of captured launches is scaled by this run's bytes per launch
    assert bench.measured_traffic("k_tail", "x", 1000.0)[0] == 1250.0
    assert bench.measured_traffic("k_tail", "x")[0] is None


def test_committed_traffic_record_is_machine_readable():
    """profiles/traffic.json: one entry per kernel/workload, each with the
    sources' hash, the DRAM bytes per launch and the command that made it."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    entries = json.load(open(path))
    assert entries
    for k, e in entries.items():
        assert "/" in k
        assert len(e["kernel_source_sha256"]) == 64
        assert e.get("traffic_bytes_per_launch", 0) > 0 or e["dram_per_algorithmic_byte"] > 0
        assert "ncu" in e["command"] and "--clock-control none" in e["command"]


def test_algorithmic_bytes_per_unit():
    sys.path.insert(0, ROOT)
    import bench
    info = {"out_scanned": 10, "front_visits": 2, "in_scanned": 100, "active_visits": 3}
    assert bench.alg_bytes(info) == (16 * 10 + 36 * 2, 24 * 100 + 48 * 3)


def test_window_width_default_and_rule_bits():
    """The windowed rules take --delta, else max weight / maximum out-degree
    (at least 1); their rule bits are the library's."""
    sys.path.insert(0, ROOT)
    import bench
    import graphgen as gg
    import paper_1812_10499_gb300 as P
    g = gg.grid(40, 30, 1, 10000, 1)                       # max out-degree 4
    assert bench.window_delta(g, None) == round(int(g.w.max()) / 4)
    assert bench.window_delta(g, 77) == 77
    assert bench.window_delta(gg.rmat(12, 16, 1, 255, 2), None) == 1   # hubs: window 1
    for name in ("thr-win", "mind-win", "thr-cheap-win"):
        assert bench.RULES[name] & P.SSSP_RULE_WINDOWED
        assert not bench.RULES[name] & P.SSSP_RULE_LABEL_CORRECTING


def test_kernel_hash_ignores_comments_and_layout():
    """The profiles' source hash follows the code only: comments and spacing
    do not change it, a code token does; literals are kept whole."""
    sys.path.insert(0, ROOT)
    import bench
    a = "int f(int x) {  // add one\n    return x + 1; /* done */ }\n"
    b = "int f(int x) {\n  return x + 1;\n}\n"
    assert bench._code_only(a) == bench._code_only(b) == "int f(int x) { return x + 1; }"
    assert bench._code_only("return x + 2;") != bench._code_only("return x + 1;")
    assert bench._code_only('const char* s = "a // b /* c */";') == 'const char* s = "a // b /* c */";'
    assert bench._code_only("char q = '\"'; // x") == "char q = '\"';"


def test_cpu_baseline_legs():
    """The CPU legs time the oracle as it stands: Dijkstra on one thread, and
    Round R one query per core in spawned processes that build their own
    graphs from the seeds."""
    sys.path.insert(0, ROOT)
    import bench
    import graphgen as gg
    g = gg.random_graph(2000, 6, 1, 50, 5)
    gteps, used, secs = bench.cpu_dijkstra_gteps(g, [0, 1, 2], 60.0)
    assert gteps > 0 and used == 3 and secs > 0
    tasks = [("var", 1500 + 10 * i, 7000 + i, i) for i in range(6)]
    tasks += [("rmat", 10, 3, s) for s in (0, 1)]
    qps, done, busy, cores = bench.cpu_queries_per_s(tasks, 120.0, cores=2)
    assert done == 8 and cores == 2 and busy > 0 and qps > 0
    res, cores = bench.oracle_sample(tasks[:3], cores=2)
    assert cores == 2 and len(res) == 3
    import oracle
    for (secs, d, r), (_, n, gseed, s) in zip(res, tasks[:3]):
        ref = oracle.round_r(gg.random_var_graph(n, 4, 16, 1, 1000, gseed), s)
        assert secs > 0 and np.array_equal(d, ref.dist) and r == ref.rounds
