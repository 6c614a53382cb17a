"""Host-side logic of the autotuner: candidate set and the on-disk cache."""
import numpy as np

from paper_2602_08501_gb300 import autotune


class _FakeCode:
    n = 64
    n_patterns = 3
    frozen = np.zeros(64, np.uint8)
    patterns = np.arange(3, dtype=np.uint64).reshape(3, 1)


def test_candidates_cover_no_split_and_sm_multiples():
    c = autotune.candidates(152)
    assert c[0] == 0 and 76 in c and 152 in c and 304 in c and c == sorted(set(c))


def test_cache_roundtrip_and_key(tmp_path, monkeypatch):
    monkeypatch.setenv("MPWSD_TUNE_CACHE", str(tmp_path / "t.json"))
    k1 = autotune.tune_key(_FakeCode(), 8, 4, [256, 2048], "NVIDIA GB300", 152)
    k2 = autotune.tune_key(_FakeCode(), 16, 4, [256, 2048], "NVIDIA GB300", 152)
    assert k1 != k2 and "L8" in k1 and "152sm" in k1
    autotune._store_cache(autotune.cache_path(), {k1: {"value": 76, "times_ms": {"0": 1.0}}})
    assert autotune._load_cache(autotune.cache_path())[k1]["value"] == 76
    assert autotune._load_cache(str(tmp_path / "missing.json")) == {}


def test_two_pass_search_finds_the_best_shape_then_split():
    # a separable cost with its minimum at shape 2, split 76
    cost = {0: 10.0, 1: 10.5, 2: 9.0, 3: 9.5}
    calls = []

    def run(shape, split):
        calls.append((shape, split))
        return cost[shape] + abs(split - 76) * 0.01

    sh, sp = autotune.choose([0, 1, 2, 3], autotune.candidates(152), 76, run)
    assert (sh, sp) == (2, 76)
    # the split sweep only ran for the chosen shape
    assert {s for s, v in calls if v not in (0, 76)} == {2}
    # ties go to the lower shape and split
    assert autotune.choose([0, 1], [0, 38], 38, lambda a, b: 1.0) == (0, 0)
