"""GPU parity of the tcgen05 BF16 hi+lo scoring path against the FP64 oracle.

The scoring step alone: approximate scores within the stated margin of the
oracle's gains (Eq. (5)) and the exact minimum recoverable. Whole decodes:
bit-exact against the oracle and identical to the FP32 CUDA-core form."""
import numpy as np
import pytest

import synth
from gpu_common import FLAG_PARITY_MASK, cuda_or_skip, oracle_code, to_words, torch
from test_gpu_parity import _decode_parity, _dev, _score_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    return cuda_or_skip()


@pytest.fixture(scope="module")
def rm26(mp):
    return mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16])


@pytest.fixture(scope="module")
def rm26_or(oracle_mod):
    return oracle_code(oracle_mod, 6, 2, 6, [16])


@pytest.mark.parametrize("M", [1, 7, 128, 129, 300, 1000])
def test_tc_score_topk_rm26(mp, rm26, rm26_or, oracle_mod, M):
    """2604 patterns = 10 full 256-pattern tiles + a ragged one; M spans row-block tails."""
    _score_case(mp, rm26, rm26_or, oracle_mod, "bf16x2", M, seed=1000 + M)


def test_tc_score_topk_small_pattern_set(mp, oracle_mod):
    """Fewer patterns than one tile (and than K for one case)."""
    ocode = oracle_mod.rm_code(6, 2)
    pats = ocode.enumerate_codewords([16])
    for P in (3, 100, 256, 257):
        code = mp.Code(64, ocode.frozen, 22, 0, 0, pats[:P])
        _score_case(mp, code, ocode.with_patterns(pats[:P]), oracle_mod, "bf16x2", 200, seed=P)


def test_tc_score_topk_rm27(mp, oracle_mod):
    code = mp.Code.rm(7, 2, crc_poly=0x21, crc_len=6, weights=[32])
    ocode = oracle_code(oracle_mod, 7, 2, 6, [32])
    _score_case(mp, code, ocode, oracle_mod, "bf16x2", 260, seed=27)


def test_tc_scores_close_to_fp32(mp, rm26):
    """Both kernels approximate the same scores; their kept values agree within 2 eps."""
    rng = np.random.default_rng(5)
    B, M = 64, 4096
    y = synth.grid_quantize(rng.standard_normal((B, 64)) * 1.25)
    frame = rng.integers(0, B, M).astype(np.int32)
    cw = rm26.patterns[rng.integers(0, rm26.n_patterns, M)].copy()
    args = (_dev(y), _dev(frame, torch.int32), _dev(cw.view(np.int64), torch.int64))
    v1, i1 = rm26.score_topk(*args, score_mode="bf16x2")
    v2, i2 = rm26.score_topk(*args, score_mode="fp32")
    torch.cuda.synchronize()
    l1 = np.abs(y.astype(np.float64)).sum(axis=1)[frame]
    assert np.all(np.abs(v1.cpu().numpy()[:, 0] - v2.cpu().numpy()[:, 0]) <= 2 * 2.0 ** -14 * l1)


@pytest.mark.parametrize("ebn0", [1.0, 2.0, 3.0])
def test_decode_parity_cfg1_bf16x2(mp, rm26, rm26_or, ebn0):
    wl = synth.make_workload("rm26_crc6", ebn0, 10000, seed=0)
    cw, fl, _ = _decode_parity(mp, rm26, rm26_or, wl, 8, 4, "bf16x2")
    # the two scoring forms reach identical decisions
    cw2, fl2 = rm26.decode(_dev(wl.y), 8, 4, score_mode="fp32")
    torch.cuda.synchronize()
    assert np.array_equal(cw, to_words(cw2))
    assert np.array_equal(fl & FLAG_PARITY_MASK, fl2.cpu().numpy().view(np.uint16) & FLAG_PARITY_MASK)


def test_decode_edge_cases_bf16x2(mp, rm26, rm26_or):
    n = 64
    rng = np.random.default_rng(8)
    wl = synth.make_workload("rm26_crc6", 1.0, 40, seed=12)
    for y in (wl.y[:1], wl.y[:13], np.zeros((4, n), np.float32),
              synth.grid_quantize(np.sign(rng.standard_normal((9, n))) * 20.0),
              synth.grid_quantize(rng.standard_normal((11, n)) * 2e-5)):
        sub = synth.Workload(code="rm26_crc6", n=n, k=22, k_info=16, crc_poly=0x21, crc_len=6, ebn0_db=None,
                             sigma=None, seed=0, first_frame=0, y=np.ascontiguousarray(y, np.float32), cw=None, msg=None)
        for L, T, aom in [(8, 4, False), (1, 1, True), (32, 15, True)]:
            _decode_parity(mp, rm26, rm26_or, sub, L, T, "bf16x2", aom=aom)


@pytest.mark.parametrize("ebn0", [0.5, 1.5, 2.5])
def test_decode_rm27_bf16x2(mp, oracle_mod, ebn0):
    """RM(2,7)+CRC-6 at each Eb/N0 of its workload, L = 16, T = 6, 10668 weight-32
    patterns (oracle-sized samples of the seed-2 stream)."""
    code = mp.Code.rm(7, 2, crc_poly=0x21, crc_len=6, weights=[32])
    ocode = oracle_code(oracle_mod, 7, 2, 6, [32])
    wl = synth.make_workload("rm27_crc6", ebn0, 400, seed=2)
    _, fl, _ = _decode_parity(mp, code, ocode, wl, 16, 6, "bf16x2")
    assert np.any(fl & 1)


def test_decode_cfg4_patterns_bf16x2(mp, oracle_mod):
    """Weight-16 and weight-24 patterns (294,252), L = 32, T = 8 on 400 frames of
    the seed-3 stream at 0.5 dB; both scoring forms."""
    code = mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16, 24])
    ocode = oracle_code(oracle_mod, 6, 2, 6, [16, 24])
    wl = synth.make_workload("rm26_crc6", 0.5, 400, seed=3)
    _, fl, _ = _decode_parity(mp, code, ocode, wl, 32, 8, "bf16x2")
    assert np.sum(fl & 1) >= 100
    _decode_parity(mp, code, ocode, wl, 32, 8, "fp32")


def test_tc_resolution_on_built_ties(mp, oracle_mod):
    """Rows built to tie (+-1/2 on the union of two patterns, so their scores are
    equal; y = 0, so every pattern ties): the resolved entry is the lowest index
    among the exact minima with its exact score, or, when four candidate groups
    share the band, a full list whose values lie within eps of their patterns'
    exact scores."""
    code = mp.Code.rm(6, 2, weights=[16])
    ocode = oracle_code(oracle_mod, 6, 2, 0, [16])
    n, B, M = 64, 40, 600
    rng = np.random.default_rng(97)
    y = synth.grid_quantize(rng.standard_normal((B, n)) * 1.3 + 0.2)
    P = oracle_mod.unpack_bits(ocode.patterns, n)
    for f, (p, q) in enumerate([(0, 1), (3, 40), (P.shape[0] - 1, 5), (7, 8), (100, 2000)]):
        y[f] = np.where((P[p] | P[q]) == 1, -0.5, 0.5)
    y[5] = 0.0
    frame = rng.integers(0, B, M).astype(np.int32)
    frame[:6] = np.arange(6)
    centres = np.zeros((M, code.W), np.uint64)
    for i in range(6, M):
        for p in rng.integers(0, P.shape[0], 2):
            centres[i] ^= ocode.patterns[p]
    vals, idx = code.score_topk(_dev(y), _dev(frame, torch.int32), _dev(centres.view(np.int64), torch.int64), "bf16x2")
    torch.cuda.synchronize()
    vals, idx = vals.cpu().numpy(), idx.cpu().numpy()
    fulls = 0
    for i in range(M):
        yy = y[frame[i]].astype(np.float64)
        S = -ocode.gains(yy, oracle_mod.unpack_bits(centres[i], n)) / 2.0
        eps = 2.0 ** -14 * np.abs(yy).sum()
        cnt = int(np.sum(idx[i] >= 0))
        if cnt == 4 and vals[i, 3] <= vals[i, 0] + 2 * eps:
            fulls += 1
            assert np.all(np.abs(vals[i] - S[idx[i]]) <= eps + 1e-12)
            continue
        want = int(np.flatnonzero(S == S.min())[0])
        assert cnt == 1 and idx[i, 0] == want, (i, idx[i], want)
        assert abs(vals[i, 0] - S.min()) <= 1e-6 * max(1.0, abs(S.min()))
    assert fulls >= 1  # the y = 0 row fills the list
