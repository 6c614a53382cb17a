"""Continuous stage-2 batching (mpwsd_pool_*): frames submitted in several
batches, interleaved with steps, come out bit for bit as one mpwsd_decode of
all of them (which the parity tests hold to the oracle); each frame's done
entry names the submission (stage-1 frames) or the step in which it finished,
no later than T steps after its submission; the rows the pool scores equal the
decode's; a submission beyond the free slots is refused."""
import numpy as np
import pytest

import synth
from gpu_common import cuda_or_skip, to_words, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    return cuda_or_skip()


def _run_pool(pool, y, plan, W):
    """plan: list of ('submit', nframes) / ('step', k); returns cw, fl, done and
    the step count before each submission."""
    B = y.shape[0]
    cw = torch.full((B, W), -1, dtype=torch.int64, device="cuda")
    fl = torch.full((B,), -1, dtype=torch.int16, device="cuda")
    done = torch.zeros((B,), dtype=torch.int32, device="cuda")
    lo = 0
    sub_at = []
    for op, k in plan:
        if op == "submit":
            hi = min(B, lo + k)
            sub_at.append((lo, hi, pool.steps))
            pool.submit(y[lo:hi], cw[lo:hi], fl[lo:hi], done[lo:hi])
            lo = hi
        else:
            for _ in range(k):
                pool.step()
    assert lo == B
    for _ in range(pool.T):  # drain: every trajectory ends within T steps of its submission
        pool.step()
    torch.cuda.synchronize()
    return to_words(cw), fl.cpu().numpy().view(np.uint16), done.cpu().numpy(), sub_at


@pytest.mark.parametrize("mode,use_graph", [("bf16x2", True), ("bf16x2", False), ("fp32", True)])
def test_pool_equals_one_batch_decode_rm26(mp, mode, use_graph):
    code = mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16])
    wl = synth.make_workload("rm26_crc6", 1.0, 9000, seed=81)
    y = torch.from_numpy(wl.y).cuda()
    L, T = 8, 4
    code.reset_stats()
    ref_cw, ref_fl = code.decode(y, L, T, score_mode=mode)
    torch.cuda.synchronize()
    ref_evals = code.stats()["pattern_evals"]
    ref_cw, ref_fl = to_words(ref_cw), ref_fl.cpu().numpy().view(np.uint16)
    pool = code.pool(6000, L, T, score_mode=mode, use_graph=use_graph)
    code.reset_stats()
    plan = [("submit", 3000), ("step", 1), ("submit", 1), ("step", 2), ("submit", 2500), ("step", 1),
            ("submit", 499), ("step", 3), ("submit", 3000)]
    cw, fl, done, sub_at = _run_pool(pool, y, plan, code.W)
    st = code.stats()
    assert np.array_equal(cw, ref_cw) and np.array_equal(fl, ref_fl)
    # the pool scores exactly the rows the one-batch decode scores
    assert st["pattern_evals"] == ref_evals and st["frames"] == 9000
    for s, (lo, hi, k0) in enumerate(sub_at):
        d = done[lo:hi]
        s1 = (fl[lo:hi] & 1) == 0
        assert np.all(d[s1] == -(s + 1))
        # a frame of this submission finishes in one of the T steps after it
        assert np.all((d[~s1] > k0) & (d[~s1] <= k0 + T)), s
        # ... in the step of its last iteration, or the one before it when its
        # longest trajectory was a twin retired there (its iteration count then
        # includes the step Algorithm 1 would still have run)
        it = ((fl[lo:hi][~s1] >> 4) & 15).astype(np.int32)
        assert np.all((d[~s1] >= k0 + it - 1) & (d[~s1] <= k0 + it))


def test_pool_rm27_osd_and_always_on(mp):
    code = mp.Code.rm(7, 2, weights=[32])  # RM(128, 29), no CRC: every frame goes to stage 2
    wl = synth.make_workload("rm27", 1.0, 1200, seed=82)
    y = torch.from_numpy(wl.y).cuda()
    L, T = 16, 4
    ref_cw, ref_fl = code.decode(y, L, T, osd_order=2, always_on=True)
    torch.cuda.synchronize()
    pool = code.pool(1200, L, T, always_on=True, osd_order=2)
    cw, fl, done, _ = _run_pool(pool, y, [("submit", 700), ("step", 2), ("submit", 500)], code.W)
    assert np.array_equal(cw, to_words(ref_cw)) and np.array_equal(fl, ref_fl.cpu().numpy().view(np.uint16))
    assert np.all(done >= 1)


def test_pool_refuses_beyond_its_slots_and_frees_them(mp):
    code = mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16])
    L, T = 8, 4
    pool = code.pool(1000, L, T)
    wl = synth.make_workload("rm26_crc6", 1.0, 1600, seed=83)
    y = torch.from_numpy(wl.y).cuda()
    cw = torch.empty((1600, 1), dtype=torch.int64, device="cuda")
    fl = torch.empty((1600,), dtype=torch.int16, device="cuda")
    assert pool.free_frames() == 1000
    pool.submit(y[:800], cw[:800], fl[:800])
    assert pool.free_frames() == 200
    with pytest.raises(mp.MpwsdError) as ei:
        pool.submit(y[800:1600], cw[800:1600], fl[800:1600])
    assert ei.value.status == mp.ENOMEM
    for k in range(T):
        assert pool.free_frames() == 200
        pool.step()
    assert pool.free_frames() == 1000  # T steps after a submission its slots are free again
    pool.submit(y[800:1600], cw[800:1600], fl[800:1600])
    for _ in range(T):
        pool.step()
    torch.cuda.synchronize()
    ref_cw, ref_fl = code.decode(y, L, T)
    torch.cuda.synchronize()
    assert torch.equal(cw, ref_cw) and torch.equal(fl, ref_fl)
