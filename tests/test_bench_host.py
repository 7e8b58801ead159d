"""Host-side logic of bench.py (no GPU): the work count behind the roofline, and the rule that
recorded ncu counters are reported only for kernels whose sources are unchanged since the capture."""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_window_counts_match_brute_force():
    b = _bench()
    for H, W, S in [(7, 9, 3), (12, 5, 11), (16, 16, 21)]:
        R = (S - 1) // 2
        ref = np.zeros((H, W))
        for i in range(H):
            for j in range(W):
                ref[i, j] = sum(1 for y in range(i - R, i + R + 1) for x in range(j - R, j + R + 1)
                                if 0 <= y < H and 0 <= x < W)
        assert np.array_equal(b.window_counts(H, W, S), ref)


def test_flop_counts_follow_the_stated_convention():
    b = _bench()
    n = np.array([[441.0, 121.0]])
    it = np.array([[300.0, 10.0]])
    d = 49
    want = sum((8 * nn * d + 4 * nn) * t + 5 * nn * d + 3 * nn for nn, t in [(441, 300), (121, 10)])
    assert b.nlem_flops(n, it, d) == want
    assert b.em_flops(np.array([300, 7]), 441, 49) == sum((8 * 441 * 49 + 4 * 441) * t + 2 * 441 * 49 for t in (300, 7))


def test_counters_reported_only_for_unchanged_sources(monkeypatch):
    b = _bench()
    for k in b.KERNEL_SOURCES:
        h = b.kernel_sources_hash(k)
        assert len(h) == 16 and int(h, 16) >= 0
    good = {k: dict(v) for k, v in b.PROFILED.items()}
    kernel = next(iter(b.KERNEL_SOURCES))
    good[kernel] = {"sources": b.kernel_sources_hash(kernel), "traffic": 123, "fma_pipe_pct": 1.0}
    monkeypatch.setattr(b, "PROFILED", good)
    assert b.profiled_counters()[kernel] == {"traffic": 123, "fma_pipe_pct": 1.0}
    stale = dict(good)
    stale[kernel] = dict(good[kernel], sources="0" * 16)
    monkeypatch.setattr(b, "PROFILED", stale)
    assert kernel not in b.profiled_counters()


def test_source_hash_ignores_comments_and_whitespace():
    b = _bench()
    assert b._code_only("int a; // note\n  /* block\n comment */ float b;\n\n") == "int a; float b;"
    assert b._code_only("x = 1; // one") == b._code_only("x =\t1;\n")
    assert b._code_only("x = 1;") != b._code_only("x = 2;")


def test_irls_flop_count_follows_the_stated_convention():
    b = _bench()
    n = np.array([[441.0, 121.0]])
    d = 49
    want = sum((5 * nn * d + 4 * nn) * 4 + 5 * nn * d + 3 * nn for nn in (441, 121))
    assert b.irls_flops(n, 4, d) == want


def test_fast_flop_count_follows_the_stated_convention():
    # 10 flops per element and iteration, 4 per point, 5 per element on each check iteration (the W2
    # pass issues an FADD and two FFMAs per element); runs stop at check points or at the cap, so a
    # run of t iterations checked every 10 has ceil(t / 10) check iterations
    b = _bench()
    n = np.array([[441.0, 121.0]])
    it = np.array([[300.0, 20.0]])
    d = 49
    want = sum((10 * nn * d + 4 * nn) * t + 5 * nn * d * c + 5 * nn * d + 3 * nn
               for nn, t, c in [(441, 300, 30), (121, 20, 2)])
    assert b.fast_nlem_flops(n, it, d, 10) == want
    assert b.fast_em_flops(np.array([90, 300, 7]), 441, 49, 10) == sum(
        (10 * 441 * 49 + 4 * 441) * t + 5 * 441 * 49 * c + 2 * 441 * 49 for t, c in ((90, 9), (300, 30), (7, 1)))


def test_profile_cases_are_the_documented_ones():
    b = _bench()
    import inspect
    doc = inspect.getdoc(b.profile_case)
    for case in ("traffic", "bf16", "features", "irls", "color", "sets"):
        assert f"{case}:" in doc
