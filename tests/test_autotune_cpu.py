"""Autotuner host logic: batch signatures, candidate choice and the JSON cache
(with a stand-in timer; no GPU)."""
import json

from paper_1705_08266_gb300 import autotune as A


def _descs():
    return [(512, 700, 4, "cdf97", "float32", 0), (65, 4096, 1, "legall53", "int32", 1),
            (3000, 2000, 6, "cdf97", "float32", 0)]


def test_signature_order_independent_and_class_based():
    d = _descs()
    assert A.signature(d) == A.signature(list(reversed(d)))
    # same power-of-two classes -> same signature
    d2 = [(600, 900, 4, "cdf97", "float32", 0)] + d[1:]
    assert A.signature(d2) == A.signature(d)
    # another class, level count, direction or type -> another signature
    for change in [(1100, 700, 4, "cdf97", "float32", 0), (512, 700, 5, "cdf97", "float32", 0),
                   (512, 700, 4, "cdf97", "float32", 1), (512, 700, 4, "cdf97", "float16", 0)]:
        assert A.signature([change] + d[1:]) != A.signature(d)


def test_pick_fastest_and_cache(tmp_path):
    path = str(tmp_path / "tune.json")
    calls = []

    def measure(t):
        calls.append(t)
        if t["fuse_first"] == 1 and t["min_segment"] == 8:
            return None  # candidate not applicable
        return 1.0 + abs(t["warps_per_sm"] - 32) / 10 + (0.5 if t["fuse_first"] == 1 else 0)

    best = A.pick("sig", measure, cache_path=path)
    assert best["warps_per_sm"] == 32 and best["fuse_first"] == 2
    assert len(calls) == len(A.CANDIDATES)
    data = json.load(open(path))
    assert data["nonsep_reduced:sig"]["tuning"] == best
    # second call: from the cache, nothing measured
    calls.clear()
    assert A.pick("sig", measure, cache_path=path) == best
    assert calls == []
    # another scheme is another entry
    A.pick("sig", measure, cache_path=path, scheme="separable")
    assert len(calls) == len(A.CANDIDATES)


def test_corrupt_cache_is_ignored(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    best = A.pick("s", lambda t: float(t["warps_per_sm"]), cache_path=str(path))
    assert best["warps_per_sm"] == 12
    assert "nonsep_reduced:s" in json.loads(path.read_text())


def test_context_separates_cache_entries(tmp_path):
    """A tuning measured on another device or library build is not reused."""
    path = str(tmp_path / "tune.json")
    calls = []

    def measure(t):
        calls.append(t)
        return float(t["warps_per_sm"])

    A.pick("sig", measure, cache_path=path, context="GPU-A/152sm/lib1")
    n = len(calls)
    A.pick("sig", measure, cache_path=path, context="GPU-A/152sm/lib1")
    assert len(calls) == n  # cached
    A.pick("sig", measure, cache_path=path, context="GPU-B/132sm/lib1")
    assert len(calls) == 2 * n  # measured again
    assert len(json.load(open(path))) == 2
