"""The C-ABI library builds, loads and exports what include/sssp.h declares;
host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sssp.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1812_10499_gb300 import build
    import paper_1812_10499_gb300 as P
    build.build()
    return P.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(sssp_\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sssp_create", "sssp_solve", "sssp_solve_device", "sssp_solve_batch",
                     "sssp_serve_open", "sssp_serve_submit", "sssp_serve_poll",
                     "sssp_destroy", "sssp_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    so = os.path.join(ROOT, "paper_1812_10499_gb300", "libsssp.so")
    out = subprocess.check_output(["nm", "-D", "--defined-only", so], text=True)
    exported = set(re.findall(r" T (sssp_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_library_targets_sm_103a():
    src = open(os.path.join(ROOT, "paper_1812_10499_gb300", "build.py")).read()
    assert "arch=compute_103a,code=sm_103a" in src


def test_strerror(lib):
    import paper_1812_10499_gb300 as P
    assert P.sssp_strerror(0) == "ok"
    assert "positive" in P.sssp_strerror(-2)
    assert P.sssp_strerror(12345) == "unknown status"


def _create(n, row_ptr, col, w):
    import paper_1812_10499_gb300 as P
    lib = P.load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.uint64)
    col = np.ascontiguousarray(col, dtype=np.uint32)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    h = ctypes.c_void_p()
    return lib.sssp_create(n, int(row_ptr[-1]), row_ptr.ctypes.data,
                           col.ctypes.data if len(col) else None,
                           w.ctypes.data if len(w) else None, None, None, None, None,
                           ctypes.byref(h))


def test_create_rejects_bad_graphs_before_touching_a_device(lib):
    # Sec. I: weights must be strictly positive.
    assert _create(3, [0, 1, 2, 2], [1, 2], [5, 0]) == -2
    # Target out of range.
    assert _create(3, [0, 1, 2, 2], [1, 3], [5, 1]) == -1
    # Non-monotone offsets / wrong total.
    assert _create(3, [0, 2, 1, 2], [1, 2], [5, 1]) == -1
    assert _create(3, [1, 1, 2, 2], [1, 2], [5, 1]) == -1
    # n = 0.
    assert _create(0, [0], [], []) == -1
    # n * max weight must fit below the packed infinity: n = 2^20 + 1 leaves
    # 43 distance bits, and 2^20 * (2^32 - 1) does not fit.
    n = (1 << 20) + 1
    rp = np.zeros(n + 1, dtype=np.uint64)
    rp[1:] = 1
    assert _create(n, rp, [1], [0xFFFFFFFF]) == -4


def test_layout_option_checked_on_the_host(lib):
    import paper_1812_10499_gb300 as P
    rp = np.array([0, 1, 1], dtype=np.uint64)
    col = np.array([1], dtype=np.uint32)

    def create(w, layout):
        o = P.sssp_options_default()
        o.layout = layout
        wa = np.array([w], dtype=np.uint32)
        h = ctypes.c_void_p()
        return lib.sssp_create(2, 1, rp.ctypes.data, col.ctypes.data, wa.ctypes.data, None,
                               None, None, ctypes.byref(o), ctypes.byref(h))
    # Unknown layout.
    assert create(5, 3) == -1
    # Compact records need n * max weight < 2^31 - 1: 2 * 2^30 does not fit.
    assert create(1 << 30, P.SSSP_LAYOUT_COMPACT) == -4
    assert lib.sssp_layout(None) == 0


def test_rule_bits_checked_on_the_host(lib):
    import paper_1812_10499_gb300 as P
    rp = np.array([0, 1, 1], dtype=np.uint64)
    col = np.array([1], dtype=np.uint32)
    wa = np.array([3], dtype=np.uint32)

    def create(rule, delta=0):
        o = P.sssp_options_default()
        o.rule = rule
        o.delta = delta
        h = ctypes.c_void_p()
        return lib.sssp_create(2, 1, rp.ctypes.data, col.ctypes.data, wa.ctypes.data, None,
                               None, None, ctypes.byref(o), ctypes.byref(h))
    # An unknown bit, and windowed with label-correcting relaxation.
    assert create(8) == -1
    assert create(P.SSSP_RULE_WINDOWED | P.SSSP_RULE_LABEL_CORRECTING, 5) == -1
    # Predecessor counts are label-setting only.
    assert create(P.SSSP_RULE_PRED_COUNT | P.SSSP_RULE_LABEL_CORRECTING) == -1
    assert create(P.SSSP_RULE_PRED_COUNT | P.SSSP_RULE_WINDOWED, 5) == -1
    assert create(64) == -1
    # The options structure carries the window width after alloc_ctx.
    assert P.sssp_options.delta.offset == P.sssp_options.alloc_ctx.offset + 8


def test_host_alloc_arguments_checked_on_the_host(lib):
    p = ctypes.c_void_p()
    assert lib.sssp_host_alloc(0, ctypes.byref(p)) == -1
    assert lib.sssp_host_alloc(64, None) == -1
    lib.sssp_host_free(None)


def test_selftest_argument_checked_on_the_host(lib):
    assert lib.sssp_selftest_barrier_timeout(0) == -1
    assert lib.sssp_selftest_barrier_timeout(20000) == -1


def test_null_handles(lib):
    assert lib.sssp_solve(None, 0, None, None) == -1
    assert lib.sssp_solve_ex(None, 0, None, None) == -1
    assert lib.sssp_serve_poll(None, 1, None) == -1
    lib.sssp_destroy(None)


def test_product_fails_loudly_without_the_library(tmp_path):
    import paper_1812_10499_gb300 as P
    saved = P._lib
    try:
        P._lib = None
        with pytest.raises(RuntimeError):
            P.load(str(tmp_path / "missing.so"))
    finally:
        P._lib = saved


def test_binding_constants_match_the_header():
    """Every #define of include/sssp.h with a plain integer value has the
    same value in the Python binding."""
    import paper_1812_10499_gb300 as P
    text = open(HEADER).read()
    defs = re.findall(r"^#define (SSSP_\w+)\s+\(?(-?\d+)u?\)?", text, flags=re.M)
    assert len(defs) > 20
    for name, val in defs:
        if hasattr(P, name):
            assert getattr(P, name) == int(val), name
    for name in ("SSSP_E_INVAL", "SSSP_E_SOURCE_RANGE", "SSSP_RULE_WINDOWED", "SSSP_RULE_PRED_COUNT",
                 "SSSP_LAYOUT_COMPACT",
                 "SSSP_LOOP_PERSISTENT", "SSSP_PENDING"):
        assert hasattr(P, name), name
