"""CPU checks of the autotuner's result store (no GPU): results are keyed by
the workload, a stored best is found again, other workloads are not."""
import json

from paper_2211_11303_gb300 import autotune


def _result(n, best, eps=1e-4):
    return {"best": best, "results": [dict(best, factor_ms=1.0, solve_ms=2.0, total_ms=3.0, iterations=5,
                                           converged=True)],
            "workload": {"n": n, "kappa": 8.0, "leaf": 32, "eta": 2.0, "eps": eps, "nrhs": 8, "precision": "fp32"}}


def test_save_then_load_round_trip(tmp_path):
    path = str(tmp_path / "tuned.json")
    autotune.save(path, _result(24, {"tile": 64, "compress_at": 64}))
    autotune.save(path, _result(16, {"tile": 32, "compress_at": 48}))
    assert autotune.load(path, 24, 8.0, 1e-4) == {"tile": 64, "compress_at": 64}
    assert autotune.load(path, 16, 8.0, 1e-4) == {"tile": 32, "compress_at": 48}
    assert autotune.load(path, 24, 8.0, 1e-3) is None       # another eps
    assert autotune.load(path, 24, 8.0, 1e-4, "fp64") is None  # another precision
    assert autotune.load(str(tmp_path / "missing.json"), 24, 8.0, 1e-4) is None
    with open(path) as f:
        assert len(json.load(f)) == 2


def test_save_replaces_the_same_workload(tmp_path):
    path = str(tmp_path / "tuned.json")
    autotune.save(path, _result(24, {"tile": 64, "compress_at": 48}))
    autotune.save(path, _result(24, {"tile": 64, "compress_at": 64}))
    assert autotune.load(path, 24, 8.0, 1e-4) == {"tile": 64, "compress_at": 64}


def test_committed_result_names_a_candidate():
    import os
    path = os.path.join(os.path.dirname(autotune.__file__), "tuned.json")
    best = autotune.load(path, 24, 8.0, 1e-4)
    assert best in autotune.DEFAULT_CANDIDATES


def test_store_path_follows_the_environment(tmp_path, monkeypatch):
    import os
    monkeypatch.delenv("HLU_TUNED", raising=False)
    shipped = os.path.join(os.path.dirname(os.path.abspath(autotune.__file__)), "tuned.json")
    assert autotune.default_path() == shipped
    path = str(tmp_path / "mine.json")
    monkeypatch.setenv("HLU_TUNED", path)
    assert autotune.default_path() == path
    autotune.save(autotune.default_path(), _result(12, {"tile": 32, "compress_at": 32}))
    assert autotune.load(path, 12, 8.0, 1e-4) == {"tile": 32, "compress_at": 32}
    monkeypatch.setenv("HLU_TUNED", "")
    assert autotune.default_path() == shipped
