"""Pins for the oracle's stage 2 (Algorithm 1, Eqs. (4)-(5), Remark 1) and for
the two-stage decoder (Sec. III): the translation identity, monotone ED,
equality with brute-force ML when the sphere is the whole code, codeword
outputs, the tie rules, and stage-1 early termination."""
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ed(y, c):
    return float(np.sum((y - (1.0 - 2.0 * c.astype(np.float64))) ** 2))


def _frames(code, B, sigma, seed):
    rng = np.random.default_rng(seed)
    info = np.flatnonzero(code.frozen == 0)
    ys, cs = [], []
    for _ in range(B):
        u = np.zeros(code.n, np.uint8)
        u[info] = rng.integers(0, 2, info.size)
        c = code.encode(u)
        y = np.rint(((1.0 - 2.0 * c) + sigma * rng.standard_normal(code.n)) * 2 ** 19) / 2 ** 19
        ys.append(y)
        cs.append(c)
    return np.array(ys), np.array(cs)


def test_filter_size(oracle_mod):
    """m = max(10, ceil(0.02 |S_r(0)|)) (Sec. IV-A)."""
    base = oracle_mod.rm_code(6, 2)
    for P, m in [(62, 10), (2604, 53), (10668, 214), (294252, 5886), (3, 10)]:
        pats = np.zeros((P, 1), np.uint64)
        assert base.with_patterns(pats).filter_m == m


def test_translation_identity():
    """ED(c xor p) - ED(c) = -2 G(p) with G of Eq. (5), for squared ED."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        n = 64
        y = rng.standard_normal(n)
        c = rng.integers(0, 2, n).astype(np.uint8)
        p = rng.integers(0, 2, n).astype(np.uint8)
        xh = 1.0 - 2.0 * c
        G = np.sum(-2.0 * y[p == 1] * xh[p == 1])
        assert abs((_ed(y, c ^ p) - _ed(y, c)) - (-2.0 * G)) < 1e-9


def test_single_iteration_picks_lowest_index_best_gain(oracle_mod):
    """One anchor, J = 1: the hop goes to the lowest-index pattern among those
    with the largest gain, and only if that gain is positive (strict ED
    improvement). Brute force over the sphere in numpy."""
    code = oracle_mod.rm_code(5, 1)
    pats = code.enumerate_codewords([16])
    code = code.with_patterns(pats)
    P = oracle_mod.unpack_bits(pats, 32)
    ys, cs = _frames(code, 60, 1.3, seed=1)
    # also frames built to tie: y = -1/2 on the union of two patterns, +1/2 elsewhere
    tie_ys = []
    for a, b in [(0, 1), (3, 40), (10, 11)]:
        y = np.full(32, 0.5)
        y[(P[a] | P[b]) == 1] = -0.5
        tie_ys.append(y)
    for y, c in list(zip(ys, cs)) + [(t, np.zeros(32, np.uint8)) for t in tie_ys]:
        xh = 1.0 - 2.0 * c
        G = np.array([np.sum(-2.0 * y[p == 1] * xh[p == 1]) for p in P])
        best = np.flatnonzero(G == G.max())[0]
        want = c ^ P[best] if G.max() > 0 else c
        res = code.mpwsd(y, c[None, :], 1)
        assert res["cw"].tolist() == want.tolist()


def test_remark1_monotone_ed_and_anchor_bound(oracle_mod):
    code = oracle_mod.rm_code(6, 2)
    code = code.with_patterns(code.enumerate_codewords([16]))
    ys, cs = _frames(code, 25, 1.25, seed=2)
    for y in ys:
        # anchors: the stage-1 list
        ul, _ = code.scl(y, 4)
        anchors = np.array([code.encode(u) for u in ul])
        eds = []
        prev = None
        for J in range(0, 7):
            res = code.mpwsd(y, anchors[:1], J)
            e = _ed(y, res["cw"])
            if prev is not None:
                assert e <= prev[0]
                if res["cw"].tolist() != prev[1]:
                    assert e < prev[0]  # strict improvement on every hop
            prev = (e, res["cw"].tolist())
            eds.append(e)
        assert eds[0] == _ed(y, anchors[0])
        res = code.mpwsd(y, anchors, 4)
        assert _ed(y, res["cw"]) <= min(_ed(y, a) for a in anchors)


def test_ml_equality_when_sphere_is_whole_code_rm15(oracle_mod):
    """Pattern set = every nonzero codeword, J = 1: every codeword is one hop
    from any anchor (Eq. 3), so the output is the ML codeword."""
    code = oracle_mod.rm_code(5, 1)
    allc = code.enumerate_codewords(list(range(1, 33)))
    assert len(allc) == 63
    code = code.with_patterns(allc)
    ys, _ = _frames(code, 200, 1.4, seed=3)
    for y in ys:
        ml, ed_ml = code.ml(y)
        ul, _ = code.scl(y, 1)
        res = code.mpwsd(y, code.encode(ul[0])[None, :], 1)
        assert _ed(y, res["cw"]) == ed_ml
        # and through the two-stage decoder in always-on mode
        out = code.decode(y[None, :], 4, 1, aom=True, threads=1)
        assert _ed(y, oracle_mod.unpack_bits(out["cw"], 32)[0]) == ed_ml


def test_ml_equality_when_sphere_is_whole_code_rm26(oracle_mod):
    code = oracle_mod.rm_code(6, 2)
    allc = code.enumerate_codewords(list(range(1, 65)))
    assert len(allc) == 2 ** 22 - 1
    code = code.with_patterns(allc)
    ys, _ = _frames(code, 3, 1.3, seed=4)
    for y in ys:
        ml, ed_ml = code.ml(y)
        ul, _ = code.scl(y, 1)
        res = code.mpwsd(y, code.encode(ul[0])[None, :], 1)
        assert _ed(y, res["cw"]) == ed_ml


def test_decoder_outputs_are_codewords_and_not_worse_than_ml(oracle_mod):
    code = oracle_mod.rm_code(6, 2, crc_poly=0x21, crc_len=6)
    code = code.with_patterns(code.enumerate_codewords([16]))
    ys, _ = _frames(code, 6, 1.3, seed=6)
    out = code.decode(ys, 8, 4, threads=2)
    F = oracle_mod.kron_power(6).astype(np.int64)
    cw = oracle_mod.unpack_bits(out["cw"], 64)
    u = (cw.astype(np.int64) @ F) % 2
    assert not u[:, code.frozen.astype(bool)].any()
    for y, c in zip(ys, cw):
        _, ed_ml = code.ml(y)
        assert _ed(y, c) >= ed_ml


def test_stage1_early_exit_and_flags(oracle_mod):
    code = oracle_mod.rm_code(6, 2, crc_poly=0x21, crc_len=6)
    code = code.with_patterns(code.enumerate_codewords([16]))
    ys, cs = _frames(code, 300, 1.2, seed=8)
    out = code.decode(ys, 8, 4, threads=4, want_anchors=True)
    for f in range(len(ys)):
        a0 = out["anchors"][f, 0]
        fl = int(out["flags"][f])
        cw = oracle_mod.unpack_bits(out["cw"][f], 64)
        if code.crc_ok(a0):
            assert fl & 1 == 0 and cw.tolist() == a0.tolist() and (fl >> 4) == 0 and fl & 2
        else:
            assert fl & 1 == 1 and 1 <= (fl >> 4) & 15 <= 4
            assert bool(fl & 2) == code.crc_ok(cw)
    assert 0 < np.mean(out["flags"] & 1) < 1


def test_all_zero_observation_keeps_first_anchor(oracle_mod):
    """y = 0: every ED equals n, nothing strictly improves, and the final
    tie goes to the first anchor."""
    code = oracle_mod.rm_code(6, 2)
    code = code.with_patterns(code.enumerate_codewords([16]))
    rng = np.random.default_rng(1)
    info = np.flatnonzero(code.frozen == 0)
    anchors = []
    for _ in range(3):
        u = np.zeros(64, np.uint8)
        u[info] = rng.integers(0, 2, info.size)
        anchors.append(code.encode(u))
    res = code.mpwsd(np.zeros(64), np.array(anchors), 4)
    assert res["cw"].tolist() == anchors[0].tolist() and res["iters"] == 1
    res = code.mpwsd(np.zeros(64), np.array(anchors[::-1]), 4)
    assert res["cw"].tolist() == anchors[2].tolist()


def test_golden_regression(oracle_mod):
    """Oracle outputs on a fixed sample, written by tests/golden/make_golden.py
    (which calls only the oracle and the input generator)."""
    import synth

    with open(os.path.join(GOLDEN, "rm26_crc6_1db_seed0_first48.json")) as fh:
        gold = json.load(fh)
    wl = synth.make_workload(gold["code"], gold["ebn0_db"], gold["frames"], seed=gold["seed"])
    yint = np.rint(wl.y.astype(np.float64) * 2 ** 19).astype(np.int64)
    assert yint.tolist() == gold["y_int"]
    code = oracle_mod.rm_code(6, 2, crc_poly=0x21, crc_len=6)
    code = code.with_patterns(code.enumerate_codewords([16]))
    out = code.decode(wl.y, gold["L"], gold["T"], threads=2)
    assert [f"{int(w):016x}" for w in out["cw"][:, 0]] == gold["cw_hex"]
    assert out["flags"].tolist() == gold["flags"]


def test_gains_match_ed_differences(oracle_mod):
    """G(p) of Eq. (5) equals (ED(c) - ED(c xor p)) / 2 for squared ED."""
    code = oracle_mod.rm_code(6, 2)
    pats = code.enumerate_codewords([16])
    code = code.with_patterns(pats)
    P = oracle_mod.unpack_bits(pats, 64)
    ys, cs = _frames(code, 5, 1.2, seed=12)
    for y, c in zip(ys, cs):
        G = code.gains(y, c)
        for p in (0, 7, 100, 2603):
            assert G[p] == (_ed(y, c) - _ed(y, c ^ P[p])) / 2


def test_eval_counts_against_an_independent_emulation(oracle_mod):
    """evals (every active (trajectory, pattern) pair of Algorithm 1) and
    evals_distinct (the same without retired twins: rows that hopped onto the
    centre of a live, unretired, lower-numbered trajectory) against a numpy
    emulation of the stage-2 loop: exact scores of every pattern, argmin with
    the lowest index on ties, a hop on a strictly negative score, stop when no
    trajectory moved."""
    import synth

    code = oracle_mod.rm_code(6, 2, crc_poly=0x21, crc_len=6)
    pats = code.enumerate_codewords([16])
    code = code.with_patterns(pats)
    P = oracle_mod.unpack_bits(pats, 64).astype(np.float64)
    wl = synth.make_workload("rm26_crc6", 1.0, 120, seed=11)
    L, T = 8, 4
    out = code.decode(wl.y, L, T, threads=2, want_anchors=True)
    twins = 0
    for f in range(wl.y.shape[0]):
        if not out["flags"][f] & 1:
            assert out["evals"][f] == 0 and out["evals_distinct"][f] == 0
            continue
        y = wl.y[f].astype(np.float64)
        ul, _ = code.scl(y, L)
        cen = np.array([code.encode(u) for u in ul])
        act = np.ones(len(cen), bool)
        ret = np.zeros(len(cen), bool)
        ev = evd = 0
        for _ in range(T):
            moved = False
            for k in range(len(cen)):
                if not act[k]:
                    continue
                ev += P.shape[0]
                evd += 0 if ret[k] else P.shape[0]
                s = P @ (y * (1.0 - 2.0 * cen[k]))
                b = int(np.argmin(s))
                if s[b] < 0:
                    cen[k] ^= P[b].astype(np.uint8)
                    moved = True
                else:
                    act[k] = False
            for k in range(len(cen)):
                if act[k] and not ret[k] and any(not ret[k2] and np.array_equal(cen[k2], cen[k]) for k2 in range(k)):
                    ret[k] = True
                    twins += 1
            if not moved:
                break
        assert out["evals"][f] == ev, f
        assert out["evals_distinct"][f] == evd, f
    assert twins > 0  # the case the count exists for occurs in this sample


def test_retiring_twins_changes_no_output():
    """The GPU retires a trajectory that hops onto the centre of a live
    (hopped in the same iteration, or stopped there, and not itself retired)
    lower-numbered trajectory of its frame. Emulated here both ways on the
    frames of a seeded batch: the chosen codeword (smallest ED, lowest anchor on
    ties) and the iteration count (largest hop count + 1, at most T) agree."""
    import oracle
    import synth

    code = oracle.rm_code(6, 2, crc_poly=0x21, crc_len=6)
    pats = code.enumerate_codewords([16])
    P = oracle.unpack_bits(pats, 64).astype(np.float64)
    wl = synth.make_workload("rm26_crc6", 1.0, 150, seed=12)
    L, T = 8, 4

    def run(y, anchors, retire):
        cen = anchors.copy()
        act = np.ones(len(cen), bool)
        ret = np.zeros(len(cen), bool)
        hops = np.zeros(len(cen), int)
        for _ in range(T):
            for k in range(len(cen)):
                if not act[k] or ret[k]:
                    continue
                s = P @ (y * (1.0 - 2.0 * cen[k]))
                b = int(np.argmin(s))
                if s[b] < 0:
                    cen[k] ^= P[b].astype(np.uint8)
                    hops[k] += 1
                else:
                    act[k] = False
            if retire:
                for k in range(len(cen)):
                    if act[k] and not ret[k] and any(not ret[k2] and np.array_equal(cen[k2], cen[k]) for k2 in range(k)):
                        ret[k] = True
        ed = [float(np.sum((y - (1.0 - 2.0 * c)) ** 2)) for c in cen]
        best = int(np.argmin(ed))  # first minimum: lowest anchor on ties
        return cen[best].tolist(), min(T, int(hops.max()) + 1), int(ret.sum())

    retired = 0
    for y in wl.y.astype(np.float64):
        ul, _ = code.scl(y, L)
        anchors = np.array([code.encode(u) for u in ul])
        if code.crc_ok(anchors[0]):
            continue
        a = run(y, anchors, False)
        b = run(y, anchors, True)
        assert a[:2] == b[:2]
        retired += b[2]
    assert retired > 0
