"""Exact scoring of flat pattern sets (MPWSD_SCORE_FLATS) against the oracle.

Every minimum-weight codeword of RM(1, m) and RM(2, m) is a coset of a
subspace; the kernel scores all of them from Walsh-Hadamard coefficients of
z = y x(c) in integers. Checks: the kept candidate is the exact argmin of the
oracle's gains (Eq. (5)) with the lowest pattern index on ties, including
frames built to tie; whole decodes match the oracle bit for bit and equal the
tensor-core decodes; pattern sets that are not whole cosets are refused."""
import numpy as np
import pytest

import synth
from gpu_common import assert_decode_parity, cuda_or_skip, oracle_code, to_words, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    return cuda_or_skip()


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


@pytest.mark.parametrize("m,r,w,M", [(5, 1, 16, 700), (6, 2, 16, 3000), (7, 2, 32, 800)])
def test_flats_scores_are_the_exact_argmin(mp, oracle_mod, m, r, w, M):
    code = mp.Code.rm(m, r, weights=[w])
    ocode = oracle_code(oracle_mod, m, r, 0, [w])
    n = 1 << m
    rng = np.random.default_rng(90 + m)
    B = 50
    y = synth.grid_quantize(rng.standard_normal((B, n)) * 1.3 + 0.2)
    # a few frames built to tie: +-1/2 on the union of two patterns, and y = 0
    P = oracle_mod.unpack_bits(ocode.patterns, n)
    for f, (p, q) in enumerate([(0, 1), (3, 40), (P.shape[0] - 1, 5)]):
        y[f] = np.where((P[p] | P[q]) == 1, -0.5, 0.5)
    y[3] = 0.0
    frame = rng.integers(0, B, M).astype(np.int32)
    frame[:8] = np.arange(8)
    centres = np.zeros((M, code.W), np.uint64)
    for i in range(M):
        for p in rng.integers(0, P.shape[0], 2 if i >= 8 else 0):
            centres[i] ^= ocode.patterns[p]
    vals, idx = code.score_topk(_dev(y), _dev(frame, torch.int32), _dev(centres.view(np.int64), torch.int64), "flats")
    torch.cuda.synchronize()
    vals, idx = vals.cpu().numpy(), idx.cpu().numpy()
    assert np.all(idx[:, 1:] == -1) and np.all(np.isinf(vals[:, 1:]))
    for i in range(M):
        yy = y[frame[i]].astype(np.float64)
        S = -ocode.gains(yy, oracle_mod.unpack_bits(centres[i], n)) / 2.0
        want = int(np.flatnonzero(S == S.min())[0])  # lowest index among the exact minima
        assert idx[i, 0] == want, (i, idx[i, 0], want)
        assert abs(vals[i, 0] - S.min()) <= 1e-6 * max(1.0, abs(S.min()))


def test_flats_refuses_other_pattern_sets(mp):
    code = mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16, 24])  # weight 24: not cosets of subspaces
    y = torch.zeros((4, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(mp.MpwsdError) as ei:
        code.decode(y, 8, 4, score_mode="flats")
    assert ei.value.status == mp.EUNSUPPORTED
    sub = mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, patterns=code.patterns[:100])  # a partial sphere
    with pytest.raises(mp.MpwsdError):
        sub.decode(y, 8, 4, score_mode="flats")


@pytest.mark.parametrize("ebn0", [1.0, 3.0])
def test_flats_decode_parity_rm26(mp, oracle_mod, ebn0):
    code = mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16])
    ocode = oracle_code(oracle_mod, 6, 2, 6, [16])
    wl = synth.make_workload("rm26_crc6", ebn0, 10000, seed=0)
    cw, fl = code.decode(_dev(wl.y), 8, 4, score_mode="flats")
    torch.cuda.synchronize()
    cw, fl = to_words(cw), fl.cpu().numpy().view(np.uint16)
    ref = ocode.decode(wl.y, 8, 4)
    assert_decode_parity(cw, fl, ref, wl.y, label=f"flats rm26 {ebn0} dB")
    cw2, fl2 = code.decode(_dev(wl.y), 8, 4, score_mode="bf16x2")
    torch.cuda.synchronize()
    assert np.array_equal(cw, to_words(cw2)) and np.array_equal(fl, fl2.cpu().numpy().view(np.uint16))


def test_flats_decode_parity_rm27_and_rm128_29(mp, oracle_mod):
    code = mp.Code.rm(7, 2, crc_poly=0x21, crc_len=6, weights=[32])
    ocode = oracle_code(oracle_mod, 7, 2, 6, [32])
    wl = synth.make_workload("rm27_crc6", 1.5, 400, seed=2)
    cw, fl = code.decode(_dev(wl.y), 16, 6, score_mode="flats")
    torch.cuda.synchronize()
    assert_decode_parity(to_words(cw), fl.cpu().numpy().view(np.uint16), ocode.decode(wl.y, 16, 6), wl.y,
                         label="flats rm27")
    aom = mp.Code.rm(7, 2, weights=[32])
    oaom = oracle_code(oracle_mod, 7, 2, 0, [32])
    wl = synth.make_workload("rm27", 1.0, 300, seed=61)
    cw, fl = aom.decode(_dev(wl.y), 16, 4, score_mode="flats", osd_order=2, always_on=True)
    torch.cuda.synchronize()
    assert_decode_parity(to_words(cw), fl.cpu().numpy().view(np.uint16),
                         oaom.decode(wl.y, 16, 4, osd_order=2, aom=True), wl.y, label="flats RM(128,29) OSD(2)")


def test_flats_small_code_and_edge_inputs(mp, oracle_mod):
    code = mp.Code.rm(5, 1, weights=[16])  # RM(1,5): complements of dimension 1
    ocode = oracle_code(oracle_mod, 5, 1, 0, [16])
    rng = np.random.default_rng(93)
    for y in (synth.make_workload("rm15", 0.0, 500, seed=2).y, np.zeros((3, 32), np.float32),
              synth.grid_quantize(np.sign(rng.standard_normal((7, 32))) * 20.0)):
        cw, fl = code.decode(_dev(y), 8, 4, score_mode="flats", always_on=True)
        torch.cuda.synchronize()
        assert_decode_parity(to_words(cw), fl.cpu().numpy().view(np.uint16), ocode.decode(y, 8, 4, aom=True), y,
                             label="flats RM(1,5)")


def test_flats_pool_equals_decode(mp):
    code = mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16])
    wl = synth.make_workload("rm26_crc6", 1.0, 5000, seed=94)
    y = _dev(wl.y)
    ref_cw, ref_fl = code.decode(y, 8, 4, score_mode="flats")
    pool = code.pool(5000, 8, 4, score_mode="flats")
    cw = torch.empty_like(ref_cw)
    fl = torch.empty_like(ref_fl)
    pool.submit(y[:2000], cw[:2000], fl[:2000])
    pool.step()
    pool.submit(y[2000:], cw[2000:], fl[2000:])
    for _ in range(4):
        pool.step()
    torch.cuda.synchronize()
    assert torch.equal(cw, ref_cw) and torch.equal(fl, ref_fl)
