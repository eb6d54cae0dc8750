"""Host-side parts of the launch-shape autotuner: its cache file (merged writes, a damaged
file read as empty) and its candidate lists (every shape a valid launch description)."""
import json

import pytest

pytest.importorskip("torch")

from paper_2602_21242_gb300 import tune  # noqa: E402


def test_cache_store_merges_and_survives_damage(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    assert tune._load_cache(path) == {}
    tune._store(path, "a", {"shape": [0, 64, 2, 32], "ms_per_step": 1.5})
    tune._store(path, "b", {"shape": [1, 0, 1, 24], "ms_per_step": 0.2})
    data = json.load(open(path))
    assert set(data) == {"a", "b"} and data["a"]["shape"] == [0, 64, 2, 32]
    tune._store(path, "a", {"shape": [2, 0, 1, 16], "ms_per_step": 0.1})
    assert tune._load_cache(path)["a"]["shape"] == [2, 0, 1, 16] and "b" in tune._load_cache(path)
    open(path, "w").write("{not json")
    assert tune._load_cache(path) == {}
    assert not [p for p in (tmp_path / "sub").iterdir() if ".tmp" in p.name]


def test_cache_path_follows_the_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("OLBM_TUNE_CACHE", str(tmp_path / "x.json"))
    assert tune.cache_path() == str(tmp_path / "x.json")
    monkeypatch.delenv("OLBM_TUNE_CACHE")
    assert tune.cache_path().endswith("tune.json")


def test_candidate_shapes_are_launch_descriptions():
    """(kind, bx, by, rows): kind 0 shapes have bx a multiple of 32 and at most 512 threads; the
    pipeline and two-step shapes use by = 1; rows is positive everywhere."""
    lists = [tune.LATTICE_CANDIDATES, tune.PIPELINE_CANDIDATES, tune.TWO_STEP_CANDIDATES,
             tune.BATCH_CANDIDATES, tune.BATCH_PIPELINE_CANDIDATES, tune.BATCH_TWO_STEP_CANDIDATES]
    for shapes in lists:
        assert shapes and len(set(shapes)) == len(shapes)
        for kind, bx, by, rows in shapes:
            assert kind in (0, 1, 2) and rows >= 1
            if kind == 0:
                assert bx % 32 == 0 and bx * by <= 512
            else:
                assert by == 1 and bx >= 0
