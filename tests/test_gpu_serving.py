"""The continuous-batching request loop (serving.py) on a mixed two-code
Poisson stream: every frame is served, each result is the same as when the
frame is decoded in one big batch and when it is decoded alone, stage-2 rows
from several submissions share the pool steps, and the memory budget sizes the
pools (a budget that fits no pool for a code refuses that code)."""
import numpy as np
import pytest

import synth
from gpu_common import cuda_or_skip, to_words, torch

pytestmark = pytest.mark.gpu


def _setup(mp, n_each, rate, seed):
    from paper_2602_08501_gb300 import serving

    specs = {"rm26": serving.CodeSpec(mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16]), 8, 4),
             "rm27": serving.CodeSpec(mp.Code.rm(7, 2, crc_poly=0x21, crc_len=6, weights=[32]), 16, 6)}
    wls = {"rm26": synth.make_workload("rm26_crc6", (0.5, 3.0), n_each, seed=seed),
           "rm27": synth.make_workload("rm27_crc6", (0.5, 3.0), n_each, seed=seed + 1)}
    arrivals = {nm: serving.poisson_arrivals(rate / 2, n_each, seed=seed + 10 + i) for i, nm in enumerate(specs)}
    ys = {nm: torch.from_numpy(wls[nm].y).pin_memory() for nm in specs}
    return serving, specs, wls, arrivals, ys


def test_serving_results_equal_alone_and_in_one_batch():
    mp = cuda_or_skip()
    serving, specs, wls, arrivals, ys = _setup(mp, 6000, 2e6, seed=50)
    srv = serving.Server(specs, max_batch=4096, pool_frames=8192, min_batch=512, max_wait_s=100e-6)
    srv.warmup()
    res = srv.run(arrivals, ys)
    assert res.served == 12000 and res.dispatches >= 4
    for nm, sp in specs.items():
        assert np.all(np.isfinite(res.latency_s[nm])) and np.all(res.latency_s[nm] >= 0)
        y = wls[nm].y
        cw, fl = sp.code.decode(torch.from_numpy(y).cuda(), sp.L, sp.T)
        torch.cuda.synchronize()
        assert np.array_equal(res.cw[nm], to_words(cw)), nm
        assert np.array_equal(res.flags[nm], fl.cpu().numpy().view(np.uint16)), nm
        rng = np.random.default_rng(1)
        for f in rng.choice(y.shape[0], 60, replace=False):
            c1, f1 = sp.code.decode(torch.from_numpy(y[f:f + 1]).cuda(), sp.L, sp.T)
            torch.cuda.synchronize()
            assert np.array_equal(res.cw[nm][f], to_words(c1)[0]) and res.flags[nm][f] == f1.cpu().numpy().view(np.uint16)[0]
        # frames of several submissions share a step: fewer steps than one stage 2 per submission would launch
        assert 0 < res.steps[nm] and res.stage2_rows[nm] > 0
    assert res.steps["rm26"] + res.steps["rm27"] < res.dispatches * 5
    p = res.percentiles()
    assert p["p50"] <= p["p99"] < 1.0


def test_serving_admission_by_memory():
    mp = cuda_or_skip()
    serving, specs, wls, arrivals, ys = _setup(mp, 3000, 1e6, seed=60)
    stage = {nm: 2048 * sp.code.n * 4 for nm, sp in specs.items()}
    # room for pools of about 1024 frames (two per code), not the 4096 asked for
    budget = 4 * max(sp.code.pool_bytes(1024, sp.L) + stage[nm] for nm, sp in specs.items()) + 1024
    srv = serving.Server(specs, max_batch=2048, pool_frames=4096, mem_budget_bytes=budget, min_batch=256,
                         max_wait_s=100e-6, pools_per_code=2)
    assert all(2 * 256 <= v < 2 * 4096 for v in srv.slots.values()) and sum(srv.refused.values()) == 0
    res = srv.run(arrivals, ys)
    assert res.served == 6000
    for nm, sp in specs.items():
        cw, fl = sp.code.decode(torch.from_numpy(wls[nm].y).cuda(), sp.L, sp.T)
        torch.cuda.synchronize()
        assert np.array_equal(res.cw[nm], to_words(cw))
    # a budget that holds no pool refuses the code
    tiny = serving.Server(specs, max_batch=2048, pool_frames=4096, mem_budget_bytes=1 << 20, pools_per_code=2)
    assert tiny.refused == {"rm26": 2, "rm27": 2}
    with pytest.raises(RuntimeError):
        tiny.run(arrivals, ys)


@pytest.mark.parametrize("m,crc_code,weights,L,T", [(7, "rm27_crc6", [32], 16, 6), (6, "rm26_crc6", [16], 8, 4)])
def test_autotune_picks_a_candidate_and_output_is_unchanged(tmp_path, monkeypatch, m, crc_code, weights, L, T):
    mp = cuda_or_skip()
    from paper_2602_08501_gb300 import autotune

    monkeypatch.setenv("MPWSD_TUNE_CACHE", str(tmp_path / "tune.json"))
    code = mp.Code.rm(m, 2, crc_poly=0x21, crc_len=6, weights=weights)
    wl = synth.make_workload(crc_code, 1.5, 4096, seed=70)
    y = torch.from_numpy(wl.y).cuda()
    shapes = autotune.shapes(code)
    assert shapes == ([0, 1, 2, 3] if m == 6 else [0, 1])
    ref = None
    for sh in shapes:
        for v in (0, 16, 76, 152):
            code.tune_set(mp.TUNE_TC_SHAPE, sh)
            code.tune_set(mp.TUNE_SPLIT_ITEMS, v)
            cw, fl = code.decode(y, L, T)
            torch.cuda.synchronize()
            if ref is None:
                ref = (cw.clone(), fl.clone())
            assert torch.equal(cw, ref[0]) and torch.equal(fl, ref[1]), (sh, v)
    with pytest.raises(mp.MpwsdError):
        code.tune_set(mp.TUNE_TC_SHAPE, 9)
    r = autotune.tune(code, y, L, T, batch_sizes=(256, 4096), reps=3)
    assert not r["cached"] and code.tune_get(mp.TUNE_SPLIT_ITEMS) == r["value"]
    assert code.tune_get(mp.TUNE_TC_SHAPE) == r["shape"] in shapes
    assert r["times_ms"][f"{r['shape']}/{r['value']}"] <= r["default_ms"]
    assert autotune.tune(code, y, L, T, batch_sizes=(256, 4096), reps=3)["cached"]
