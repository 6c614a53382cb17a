"""Host logic of the serving loop that needs no GPU: batch-size buckets (so
that a replayed CUDA graph fits every batch), the seeded Poisson arrival
stream, and the latency percentiles of a run."""
import numpy as np
import pytest

serving = pytest.importorskip("paper_2602_08501_gb300.serving")


def test_buckets_are_the_smallest_power_of_two_multiple_of_the_floor():
    for b in (1, 255, 256, 257, 511, 512, 513, 65535, 65536):
        k = serving._bucket(b)
        assert k >= b and k >= 256
        assert k == 256 or k // 2 < b  # the smallest such size
        assert (k & (k - 1)) == 0  # 256 * 2^j
    assert serving._bucket(5, lo=4) == 8


def test_poisson_arrivals_are_seeded_increasing_and_have_the_rate():
    a = serving.poisson_arrivals(2e6, 200_000, seed=3)
    b = serving.poisson_arrivals(2e6, 200_000, seed=3)
    assert np.array_equal(a, b)
    assert np.all(np.diff(a) > 0) and a[0] > 0
    gaps = np.diff(np.concatenate([[0.0], a]))
    # exponential gaps: mean 1/rate, and the standard deviation equals the mean
    assert abs(gaps.mean() * 2e6 - 1.0) < 0.01
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.02
    assert not np.array_equal(a, serving.poisson_arrivals(2e6, 200_000, seed=4))


def test_latency_percentiles_pool_every_code():
    rng = np.random.default_rng(5)
    lat = {"a": rng.exponential(1e-3, 1000), "b": rng.exponential(2e-3, 500), "c": np.zeros(0)}
    res = serving.ServeResult(latency_s=lat, cw={}, flags={}, served=1500, wall_s=1.0, dispatches=10,
                              slots={}, refused_slots={})
    pooled = np.concatenate([lat["a"], lat["b"]])
    got = res.percentiles((50, 99))
    assert got["p50"] == float(np.percentile(pooled, 50)) and got["p99"] == float(np.percentile(pooled, 99))
    empty = serving.ServeResult(latency_s={}, cw={}, flags={}, served=0, wall_s=0.0, dispatches=0, slots={},
                                refused_slots={})
    assert empty.percentiles() == {"p50": None, "p99": None}


def test_pool_size_for_budget_halves_until_it_fits():
    class FakeCode:
        def pool_bytes(self, frames, L):
            return 1000 + frames * L * 10

    c = FakeCode()
    assert serving.pool_frames_for_budget(c, 8, 4096, None, 256) == 4096
    assert serving.pool_frames_for_budget(c, 8, 4096, 1000 + 4096 * 80, 256) == 4096
    assert serving.pool_frames_for_budget(c, 8, 4096, 1000 + 4095 * 80, 256) == 2048
    assert serving.pool_frames_for_budget(c, 8, 4096, 1000 + 300 * 80, 256) == 256
    assert serving.pool_frames_for_budget(c, 8, 4096, 1000 + 255 * 80, 256) == 0


def test_rows_per_step_pools_every_code():
    res = serving.ServeResult(latency_s={}, cw={}, flags={}, served=0, wall_s=1.0, dispatches=3, slots={},
                              refused_slots={}, steps={"a": 10, "b": 30}, stage2_rows={"a": 1000, "b": 3000})
    assert res.rows_per_step() == 100.0
    assert serving.ServeResult(latency_s={}, cw={}, flags={}, served=0, wall_s=1.0, dispatches=0, slots={},
                               refused_slots={}).rows_per_step() == 0.0
