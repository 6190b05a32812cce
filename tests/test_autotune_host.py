"""Host logic of the autotuner that needs no GPU: the result cache and
applying a configuration to an engine."""
import json

import pytest

import paper_1805_02755_gb300 as E
from paper_1805_02755_gb300 import autotune as A


def test_cached_result_is_returned_without_timing(tmp_path):
    path = tmp_path / "tune.json"
    best = {"config": {"scheduler": "hguided", "params": [1.0, 8], "devices": 1, "ctas": 0}, "ms": 0.2,
            "table": []}
    path.write_text(json.dumps({"gaussian|67108864|128": best}))

    def never():
        raise AssertionError("a cached shape must not build programs")

    got = A.autotune("gaussian", never, 67108864, 128, cache_path=str(path))
    assert got == best
    # another shape is a miss: with an empty space the search has nothing to time
    with pytest.raises(ValueError, match=r"min\(\)"):
        A.autotune("gaussian", never, 1024, 128, space=[], cache_path=str(path))


def test_unreadable_cache_is_ignored(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    # the broken file reads as an empty cache: the error is the empty search's, not the parser's
    with pytest.raises(ValueError, match=r"min\(\)"):
        A.autotune("mandelbrot", lambda: None, 1024, 256, space=[], cache_path=str(path))


class _FakeEngine:
    def __init__(self):
        self.calls = []

    def scheduler(self, kind, params):
        self.calls.append(("scheduler", kind, list(params)))
        return self

    def workers(self, d, c):
        self.calls.append(("workers", d, c))
        return self


def test_apply_sets_scheduler_and_workers():
    e = A.apply(_FakeEngine(), {"scheduler": "dynamic", "params": [256], "devices": 12, "ctas": 38})
    assert e.calls == [("scheduler", E.ECL_DYNAMIC, [256]), ("workers", 12, 38)]
    e = A.apply(_FakeEngine(), {"scheduler": "hguided", "params": [0.5, 4], "devices": 1, "ctas": 0})
    assert e.calls[0] == ("scheduler", E.ECL_HGUIDED, [0.5, 4])
