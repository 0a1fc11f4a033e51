"""The batched-tree autotuner's search, cache and key, on the CPU with a fake
timer (no GPU): the staged search visits 9 + 2 candidates and returns the
fastest, the choice is cached per shape key and reused, `force` re-tunes, an
unreadable cache is ignored, and the key separates GPUs, widths, alphabets,
sizes, tree counts and query counts."""
import json

import pytest

torch = pytest.importorskip("torch")

from paper_2505_03372_gb300 import autotune  # noqa: E402


def _batch(ntrees=8, n=1000, nq=5000, w=2, sigmas=(4, 256)):
    dt = {1: torch.uint8, 2: torch.int16, 4: torch.int32}[w]
    views = [torch.zeros(n, dtype=dt) for _ in range(ntrees)]
    sg = [sigmas[i % len(sigmas)] for i in range(ntrees)]
    q = {"tree": torch.zeros(nq, dtype=torch.int32), "kind": torch.zeros(nq, dtype=torch.uint8),
         "c": torch.zeros(nq, dtype=torch.int32), "arg": torch.zeros(nq, dtype=torch.int64)}
    return views, sg, q


class FakeTimer:
    def __init__(self):
        self.calls = []

    def __call__(self, views, sigmas, queries, cand):
        self.calls.append(dict(cand))
        return 10.0 - cand["lp_ctas_per_sm"] - (1.0 if cand["query_threads"] == 256 else 0.0) \
            - (0.5 if cand["sample_k"] == 8192 else 0.0)


def test_staged_search_finds_the_fastest_and_caches_it(tmp_path):
    path = str(tmp_path / "tune.json")
    views, sg, q = _batch()
    t = FakeTimer()
    best = autotune.tune_batch(views, sg, q, cache_path=path, timer=t, device_name="GPU-A")
    assert best == {"sample_k": 8192, "query_threads": 256, "lp_ctas_per_sm": 6}
    assert len(t.calls) == 11
    assert all(c["sample_k"] == 4096 for c in t.calls[:9])
    assert {c["sample_k"] for c in t.calls[9:]} == {2048, 8192}
    cache = json.load(open(path))
    key = autotune.shape_key(views, sg, q, "GPU-A")
    assert cache[key]["best"] == best and len(cache[key]["timings_ms"]) == 11
    # cached: no timing the second time
    t2 = FakeTimer()
    assert autotune.tune_batch(views, sg, q, cache_path=path, timer=t2, device_name="GPU-A") == best
    assert t2.calls == []
    # force re-tunes
    t3 = FakeTimer()
    autotune.tune_batch(views, sg, q, cache_path=path, timer=t3, device_name="GPU-A", force=True)
    assert len(t3.calls) == 11


def test_unreadable_cache_is_ignored(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    views, sg, q = _batch()
    t = FakeTimer()
    best = autotune.tune_batch(views, sg, q, cache_path=str(path), timer=t, device_name="GPU-A")
    assert len(t.calls) == 11 and best["lp_ctas_per_sm"] == 6
    assert autotune.shape_key(views, sg, q, "GPU-A") in json.load(open(path))


def test_shape_key_separates_shapes():
    base = autotune.shape_key(*_batch(), device_name="GPU-A")
    assert autotune.shape_key(*_batch(), device_name="GPU-B") != base
    assert autotune.shape_key(*_batch(w=1), device_name="GPU-A") != base
    assert autotune.shape_key(*_batch(sigmas=(4, 65536)), device_name="GPU-A") != base
    assert autotune.shape_key(*_batch(n=100000), device_name="GPU-A") != base
    assert autotune.shape_key(*_batch(ntrees=9), device_name="GPU-A") != base
    assert autotune.shape_key(*_batch(nq=1 << 20), device_name="GPU-A") != base
    assert autotune.shape_key(*_batch(), device_name="GPU-A") == base
