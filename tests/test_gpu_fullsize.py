"""Parity at the full batch sizes, in the launch configuration bench.py times.

Each test decodes a whole workload batch on the GPU exactly as the benchmark
step does (one mpwsd.Code.decode of the batch, BF16 hi+lo tensor-core
scoring, the benchmark's L and T) and checks a seeded sample of its frames
against the oracle, frame by frame: codewords and flags bit-exact, frames
whose FP64 decision gap is below 1e-6 ||y||^2 the only allowed exception.
The sample always includes frames that went to stage 2, so the scoring
kernel's full-size launches are what is being checked.
"""
import numpy as np
import pytest

import synth
from gpu_common import assert_decode_parity, cuda_or_skip, oracle_code, to_words, torch

pytestmark = pytest.mark.gpu


def _full_batch_sample(code_name, m, weights, ebn0, frames, seed, L, T, n_sample, crc_len=6, osd=None, aom=False):
    mp = cuda_or_skip()
    import oracle

    code = mp.Code.rm(m, 2, crc_poly=0x21 if crc_len else 0, crc_len=crc_len, weights=weights)
    wl = synth.make_workload(code_name, ebn0, frames, seed=seed)
    cw, fl = code.decode(torch.from_numpy(wl.y).cuda(), L, T, score_mode="bf16x2", osd_order=osd, always_on=aom)
    torch.cuda.synchronize()
    cw, fl = to_words(cw), fl.cpu().numpy().view(np.uint16)
    # half of the sample from the frames that ran stage 2, half from the whole batch
    rng = np.random.default_rng(seed + 1000)
    stage2 = np.flatnonzero(fl & 1)
    assert stage2.size > 0
    pick = np.unique(np.concatenate([rng.choice(stage2, n_sample // 2, replace=False),
                                     rng.choice(frames, n_sample - n_sample // 2, replace=False)]))
    ocode = oracle_code(oracle, m, 2, crc_len, weights)
    ref = ocode.decode(wl.y[pick], L, T, osd_order=osd, aom=aom)
    assert_decode_parity(cw[pick], fl[pick], ref, wl.y[pick], label=f"{code_name} {frames} frames (sample)")
    return pick.size, int(np.sum(fl[pick] & 1))


def test_rm26_1db_million_frames_sampled():
    """RM(2,6)+CRC-6, 1 dB, 10^6 frames from seed 1, L = 8, T = 4, 2604 patterns."""
    checked, s2 = _full_batch_sample("rm26_crc6", 6, [16], 1.0, 1_000_000, 1, 8, 4, 4000)
    assert checked >= 3900 and s2 >= 2000


def test_rm27_1p5db_million_frames_sampled():
    """RM(2,7)+CRC-6, 1.5 dB, 10^6 frames from seed 2, L = 16, T = 6, 10668 patterns."""
    checked, s2 = _full_batch_sample("rm27_crc6", 7, [32], 1.5, 1_000_000, 2, 16, 6, 400)
    assert checked >= 390 and s2 >= 200


def test_rm26_l32_large_sphere_sampled():
    """RM(2,6)+CRC-6, 0.5 dB, 2 x 10^5 frames from seed 3, L = 32, T = 8, 294252 patterns."""
    checked, s2 = _full_batch_sample("rm26_crc6", 6, [16, 24], 0.5, 200_000, 3, 32, 8, 200)
    assert checked >= 190 and s2 >= 100


@pytest.mark.parametrize("order", [2, 4])
def test_rm128_29_always_on_million_frames_sampled(order):
    """RM(128, 29) without CRC, stage 2 always on, OSD(order) anchors, 1 dB,
    10^6 frames from seed 6, L = 16, J = 4, 10668 patterns (the paper's RM
    pipeline as bench.py runs it)."""
    checked, s2 = _full_batch_sample("rm27", 7, [32], 1.0, 1_000_000, 6, 16, 4, 300, crc_len=0, osd=order, aom=True)
    assert checked >= 290 and s2 == checked
