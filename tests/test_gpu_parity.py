"""GPU parity: every step of the hot path through the C ABI against the FP64
oracle on the same seeded inputs.

Stage 1 (SC-list): bit-exact codewords and metrics. Scoring: the kernel's
approximate scores within the stated margin of the oracle's gains, and the
exact argmin recovered. Full decode (stage 1 + Algorithm 1 + final select):
bit-exact codewords and flags, FP32 and BF16-split scoring alike."""
import numpy as np
import pytest

import synth
from gpu_common import assert_decode_parity, cuda_or_skip, oracle_code, to_words, torch

pytestmark = pytest.mark.gpu

EPS_SCALE = 2.0 ** -14  # re-rank margin per unit of ||y||_1 (the library's kEpsScale)


@pytest.fixture(scope="module")
def mp():
    return cuda_or_skip()


@pytest.fixture(scope="module")
def rm26(mp):
    return mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16])


@pytest.fixture(scope="module")
def rm26_or(oracle_mod):
    return oracle_code(oracle_mod, 6, 2, 6, [16])


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


@pytest.mark.parametrize("L", [1, 2, 3, 5, 8, 16, 32])
def test_stage1_list_bit_exact_rm26(mp, rm26, rm26_or, oracle_mod, L):
    wl = synth.make_workload("rm26_crc6", 1.0, 301, seed=7)
    cw, pm = rm26.stage1_list(_dev(wl.y), L)
    torch.cuda.synchronize()
    cw, pm = to_words(cw), pm.cpu().numpy()
    for f in range(wl.B):
        ul, pml = rm26_or.scl(wl.y[f].astype(np.float64), L)
        want = oracle_mod.pack_bits(np.array([rm26_or.encode(u) for u in ul]))
        assert np.array_equal(cw[f, :len(ul)], want), f
        assert np.array_equal(pm[f, :len(ul)], np.rint(pml * 2 ** 19).astype(np.int64)), f


@pytest.mark.parametrize("m,r,L", [(5, 1, 8), (5, 1, 32), (7, 2, 16), (7, 2, 4)])
def test_stage1_list_bit_exact_other_codes(mp, oracle_mod, m, r, L):
    code = mp.Code.rm(m, r)
    ocode = oracle_mod.rm_code(m, r)
    n = 1 << m
    rng = np.random.default_rng(m * 100 + L)
    y = synth.grid_quantize(rng.standard_normal((97, n)) * 1.3 + 0.3)
    cw, pm = code.stage1_list(_dev(y), L)
    torch.cuda.synchronize()
    cw, pm = to_words(cw), pm.cpu().numpy()
    for f in range(y.shape[0]):
        ul, pml = ocode.scl(y[f].astype(np.float64), L)
        want = oracle_mod.pack_bits(np.array([ocode.encode(u) for u in ul]))
        assert np.array_equal(cw[f, :len(ul)], want), f
        assert np.array_equal(pm[f, :len(ul)], np.rint(pml * 2 ** 19).astype(np.int64)), f


def test_stage1_list_generic_frozen_set(mp, oracle_mod):
    """A frozen set that is not Reed-Muller takes the run-time-checked kernel."""
    rng = np.random.default_rng(4)
    n = 64
    fz = np.ones(n, np.uint8)
    fz[rng.choice(n, 20, replace=False)] = 0
    fz[n - 1] = 1  # a frozen leaf after the last information leaf: final re-sort path
    k = int((fz == 0).sum())
    ocode = oracle_mod.Code(n, fz, k)
    pats = ocode.enumerate_codewords(list(range(1, 65)))[:50]
    code = mp.Code(n, fz, k, 0, 0, pats)
    y = synth.grid_quantize(rng.standard_normal((64, n)) * 1.2)
    for L in (1, 8, 16):
        cw, pm = code.stage1_list(_dev(y), L)
        torch.cuda.synchronize()
        cw, pm = to_words(cw), pm.cpu().numpy()
        for f in range(y.shape[0]):
            ul, pml = ocode.scl(y[f].astype(np.float64), L)
            want = oracle_mod.pack_bits(np.array([ocode.encode(u) for u in ul]))
            assert np.array_equal(cw[f, :len(ul)], want), (L, f)
            assert np.array_equal(pm[f, :len(ul)], np.rint(pml * 2 ** 19).astype(np.int64)), (L, f)


def _score_case(mp, code, ocode, oracle_mod, mode, M, seed):
    rng = np.random.default_rng(seed)
    n = code.n
    B = 37
    y = synth.grid_quantize(rng.standard_normal((B, n)) * 1.25 + 0.2)
    frame = rng.integers(0, B, M).astype(np.int32)
    # centres: random codewords (XOR of a few patterns)
    P = ocode.patterns
    centres = np.zeros((M, code.W), np.uint64)
    for i in range(M):
        for p in rng.integers(0, P.shape[0], 3):
            centres[i] ^= P[p]
    vals, idx = code.score_topk(_dev(y), _dev(frame, torch.int32), _dev(centres.view(np.int64), torch.int64), mode)
    torch.cuda.synchronize()
    vals, idx = vals.cpu().numpy(), idx.cpu().numpy()
    for i in range(M):
        yy = y[frame[i]].astype(np.float64)
        G = ocode.gains(yy, oracle_mod.unpack_bits(centres[i], n))
        S = -G / 2.0
        eps = EPS_SCALE * np.abs(yy).sum()
        cnt = int(np.sum(idx[i] >= 0))
        assert cnt >= 1 and np.all(idx[i, :cnt] >= 0) and np.all(idx[i, cnt:] == -1)
        assert np.all(np.diff(vals[i, :cnt]) >= 0)
        # every kept value within eps of its exact score
        assert np.all(np.abs(vals[i, :cnt] - S[idx[i, :cnt]]) <= eps)
        full = cnt == 4 and vals[i, 3] <= vals[i, 0] + 2 * eps
        # the exact minimum is kept, unless the list is full within the margin (rescan)
        best = np.flatnonzero(S == S.min())[0]
        assert best in idx[i, :cnt] or full
        if mode == "bf16x2" and not full:
            # the tensor-core form resolves its candidate groups exactly: the single
            # entry is the exact argmin (lowest index on ties) with its exact score
            assert cnt == 1 and idx[i, 0] == best, (i, idx[i], best)
            assert abs(vals[i, 0] - S.min()) <= 1e-6 * max(1.0, abs(S.min()))
            continue
        # every pattern left out is outside the band of the re-rank
        outside = np.setdiff1d(np.arange(P.shape[0]), idx[i, :cnt])
        if outside.size and not full:
            assert S[outside].min() > vals[i, 0] + 2 * eps - eps - 1e-9


@pytest.mark.parametrize("M", [1, 5, 128, 300])
def test_score_topk_fp32(mp, rm26, rm26_or, oracle_mod, M):
    _score_case(mp, rm26, rm26_or, oracle_mod, "fp32", M, seed=M)


def _decode_parity(mp, code, ocode, wl, L, T, mode, aom=False, rule="top1"):
    y = wl.y
    cw, fl = code.decode(_dev(y), L, T, score_mode=mode, always_on=aom, rule=rule)
    torch.cuda.synchronize()
    cw, fl = to_words(cw), fl.cpu().numpy().view(np.uint16)
    ref = ocode.decode(y, L, T, aom=aom, rule=1 if rule == "any" else 0)
    # bit-exact on every frame; a few near-tie frames (min decision gap < 1e-6 ||y||^2) the only allowed exception
    assert_decode_parity(cw, fl, ref, y, label=f"{wl.code} L={L} T={T} {mode} aom={aom} {rule}")
    return cw, fl, ref


@pytest.mark.parametrize("ebn0", [1.0, 2.0, 3.0])
def test_decode_parity_cfg1_fp32(mp, rm26, rm26_or, ebn0):
    """RM(2,6)+CRC-6, L = 8, T = 4, 2604 weight-16 patterns, 10^4 frames from seed 0."""
    wl = synth.make_workload("rm26_crc6", ebn0, 10000, seed=0)
    _, fl, _ = _decode_parity(mp, rm26, rm26_or, wl, 8, 4, "fp32")
    assert 0 < np.mean(fl & 1) < 1


def test_decode_edge_cases_fp32(mp, rm26, rm26_or, oracle_mod):
    n = 64
    rng = np.random.default_rng(3)
    wl = synth.make_workload("rm26_crc6", 1.0, 50, seed=11)
    cases = {
        "one_frame": wl.y[:1],
        "ragged_7": wl.y[:7],
        "zeros": np.zeros((5, n), np.float32),
        "clamp": synth.grid_quantize(np.sign(rng.standard_normal((9, n))) * 20.0),
        "noiseless": (1.0 - 2.0 * wl.cw[:12]).astype(np.float32),
        "tiny_values": synth.grid_quantize(rng.standard_normal((11, n)) * 2e-5),
    }
    for name, y in cases.items():
        sub = synth.Workload(code="rm26_crc6", n=n, k=22, k_info=16, crc_poly=0x21, crc_len=6, ebn0_db=None,
                             sigma=None, seed=0, first_frame=0, y=np.ascontiguousarray(y, np.float32), cw=None, msg=None)
        for L, T, aom in [(8, 4, False), (1, 1, True), (3, 2, True), (32, 15, False)]:
            _decode_parity(mp, rm26, rm26_or, sub, L, T, "fp32", aom=aom)
    # empty batch
    cw, fl = rm26.decode(torch.zeros((0, n), device="cuda"), 8, 4, score_mode="fp32")
    assert cw.shape[0] == 0


def test_decode_any_rule_fp32(mp, rm26, rm26_or):
    wl = synth.make_workload("rm26_crc6", 1.5, 3000, seed=5)
    _decode_parity(mp, rm26, rm26_or, wl, 8, 4, "fp32", rule="any")


def test_decode_small_code_list_longer_than_codebook(mp, oracle_mod):
    """RM(1,5) without CRC (always-on), weight-16 patterns, L = 32 < 2^6."""
    code = mp.Code.rm(5, 1, weights=[16])
    ocode = oracle_code(oracle_mod, 5, 1, 0, [16])
    wl = synth.make_workload("rm15", 0.0, 2000, seed=2)
    for L in (1, 8, 32):
        _decode_parity(mp, code, ocode, wl, L, 4, "fp32", aom=True)


def test_decode_rm27_fp32(mp, oracle_mod):
    """RM(2,7)+CRC-6, L = 16, T = 6, 10668 weight-32 patterns (oracle-sized subset)."""
    code = mp.Code.rm(7, 2, crc_poly=0x21, crc_len=6, weights=[32])
    ocode = oracle_code(oracle_mod, 7, 2, 6, [32])
    wl = synth.make_workload("rm27_crc6", 1.5, 400, seed=2)
    _decode_parity(mp, code, ocode, wl, 16, 6, "fp32")


def test_stats_counters(mp, rm26, rm26_or):
    wl = synth.make_workload("rm26_crc6", 1.0, 4000, seed=9)
    rm26.reset_stats()
    _, fl, ref = _decode_parity(mp, rm26, rm26_or, wl, 8, 4, "fp32")
    st = rm26.stats()
    assert st["frames"] == 4000
    assert st["stage2_frames"] == int(np.sum(fl & 1))
    assert st["trajectories"] == 8 * st["stage2_frames"]
    # rows the GPU scores: duplicates of a lower-numbered trajectory are retired
    assert st["pattern_evals"] == int(ref["evals_distinct"].sum())
    assert st["pattern_evals"] < int(ref["evals"].sum())
    # stage 1, T x (score, re-rank + hop, rescan), T - 1 duplicate retirements, final
    assert st["kernel_launches"] >= 1 + 3 * 4 + 3 + 1


def test_graph_replay_matches_direct_launches(mp, rm26):
    """use_graph: the first call records the launch sequence, later identical
    calls replay it; results equal the direct launches, call after call."""
    wl = synth.make_workload("rm26_crc6", 1.0, 3000, seed=41)
    y = _dev(wl.y)
    ws = rm26.workspace(4096, 8)
    cw_ref, fl_ref = rm26.decode(y, 8, 4, workspace=ws)
    cw = torch.empty_like(cw_ref)
    fl = torch.empty_like(fl_ref)
    for mode in ("bf16x2", "fp32"):
        ref = rm26.decode(y, 8, 4, score_mode=mode, workspace=ws)
        for _ in range(3):
            cw.fill_(-1)
            fl.fill_(-1)
            rm26.decode(y, 8, 4, score_mode=mode, workspace=ws, cw_out=cw, flags_out=fl, use_graph=True)
            torch.cuda.synchronize()
            assert torch.equal(cw, ref[0]) and torch.equal(fl, ref[1])
    # new input data in the same buffer: the replay reads it
    y.copy_(_dev(synth.make_workload("rm26_crc6", 2.0, 3000, seed=42).y))
    ref = rm26.decode(y, 8, 4, workspace=ws)
    rm26.decode(y, 8, 4, workspace=ws, cw_out=cw, flags_out=fl, use_graph=True)
    torch.cuda.synchronize()
    assert torch.equal(cw, ref[0]) and torch.equal(fl, ref[1])
