"""Pins for the oracle's minimum decision gap (``min_gap``), the number the
tie rule of every GPU parity test rests on.

Definition restated here (Algorithm 1 and its final step, squared ED): every
decision of a trajectory chooses among "stay" and one hop per pattern; its gap
is the difference between the two smallest squared Euclidean distances of those
candidates (0 when they tie). The final choice compares the trajectory end
points; its gap is the smallest ED excess of an end point whose codeword
differs from the chosen one. ``min_gap`` is the smallest gap over all of a
frame's decisions. The expected values below come from closed forms derived by
hand (the overlap of two weight-16 codewords of RM(2,6) is 0, 1, 2, 4, 8 or 16:
they are 4-flats of AG(6, 2)), and from a brute-force emulation that forms every
candidate codeword and measures its distance directly, so a wrong scale, a
dropped "stay" candidate or a missing final comparison fails one of them."""
import numpy as np
import pytest


def _ed(y, c):
    return float(np.sum((np.asarray(y, np.float64) - (1.0 - 2.0 * np.asarray(c, np.float64))) ** 2))


@pytest.fixture(scope="module")
def rm26(oracle_mod):
    code = oracle_mod.rm_code(6, 2)
    pats = code.enumerate_codewords([16])
    return code.with_patterns(pats), oracle_mod.unpack_bits(pats, 64)


def test_stay_decision_gap_is_the_best_hop_excess(rm26):
    """y = a on every position, anchor 0: every weight-16 hop raises the ED by
    4 * 16 * a, so the one decision stays with gap 64 a."""
    code, _ = rm26
    for a in (0.25, 0.5, 1.0, 1.375):
        res = code.mpwsd(np.full(64, a), np.zeros((1, 64), np.uint8), 1)
        assert res["cw"].tolist() == [0] * 64
        assert res["min_gap"] == 64.0 * a


@pytest.mark.parametrize("a,b", [(0.5, 1.0), (0.25, 1.5), (1.0, 0.625), (1.5, 0.5), (0.75, 0.75)])
def test_hop_decision_gap_closed_form(rm26, a, b):
    """y = -b on the support of one pattern p1 and +a elsewhere, anchor 0.
    A pattern meeting supp p1 in t positions changes the ED by
    4 (16 a - t (a + b)), so p1 (t = 16) is the hop, with ED change -64 b.
    The runner-up is the best t = 8 pattern when a < b (change 32 (a - b) < 0)
    and "stay" (change 0) otherwise: gap 32 (a + b) or 64 b. After the hop every
    z = y x is positive, the best further move costs 64 min(a, b) (a pattern
    disjoint from p1, or p1 again), so a second iteration stays with that gap."""
    code, P = rm26
    p1 = 137
    y = np.where(P[p1] == 1, -b, a)
    res1 = code.mpwsd(y, np.zeros((1, 64), np.uint8), 1)
    assert res1["cw"].tolist() == P[p1].tolist()
    gap1 = 32.0 * (a + b) if a < b else 64.0 * b
    assert res1["min_gap"] == gap1
    res2 = code.mpwsd(y, np.zeros((1, 64), np.uint8), 2)
    assert res2["cw"].tolist() == P[p1].tolist() and res2["iters"] == 2
    assert res2["min_gap"] == min(gap1, 64.0 * min(a, b))


def test_two_patterns_tie_gives_zero_gap(rm26):
    """y = -1/2 on the union of two disjoint patterns, +1/2 elsewhere: both hops
    lower the ED by the same amount, so the first decision has gap 0."""
    code, P = rm26
    p1 = 0
    p2 = next(q for q in range(1, P.shape[0]) if not np.any(P[q] & P[p1]))
    y = np.where((P[p1] | P[p2]) == 1, -0.5, 0.5)
    res = code.mpwsd(y, np.zeros((1, 64), np.uint8), 1)
    assert res["cw"].tolist() == P[p1].tolist()  # lowest index among the tied hops
    assert res["min_gap"] == 0.0


def test_final_choice_gap_counts_distinct_end_points_only(rm26):
    """With no iteration (T = 0) the only decision is the final choice among
    the anchors. y = a everywhere: ED(p) - ED(0) = 64 a for a weight-16 p.
    A repeated anchor equal to the winner adds no gap; a lone anchor has none."""
    code, P = rm26
    a = 0.75
    y = np.full(64, a)
    z = np.zeros(64, np.uint8)
    res = code.mpwsd(y, np.array([P[5], z, P[9]]), 0)
    assert res["cw"].tolist() == z.tolist() and res["final_k"] == 1
    assert res["min_gap"] == 64.0 * a
    res = code.mpwsd(y, np.array([z, z]), 0)
    assert res["final_k"] == 0 and res["min_gap"] == np.inf
    res = code.mpwsd(y, z[None, :], 0)
    assert res["min_gap"] == np.inf
    # two different end points at the same distance: gap 0, lowest anchor wins
    res = code.mpwsd(y, np.array([P[9], P[5]]), 0)
    assert res["final_k"] == 0 and res["cw"].tolist() == P[9].tolist() and res["min_gap"] == 0.0


def test_zero_observation_gap_is_zero(rm26):
    code, _ = rm26
    res = code.mpwsd(np.zeros(64), np.zeros((2, 64), np.uint8), 3)
    assert res["min_gap"] == 0.0


def _emulated_min_gap(y, anchors, P, T):
    """Algorithm 1 by brute force: every candidate codeword of a decision is
    formed and its squared distance measured directly; the gap is the spread of
    the two smallest distances among stay + hops."""
    y = np.asarray(y, np.float64)
    cen = [a.copy() for a in anchors]
    active = [True] * len(cen)
    gaps = []
    for _ in range(T):
        moved = False
        for k in range(len(cen)):
            if not active[k]:
                continue
            cands = np.concatenate([cen[k][None, :], cen[k][None, :] ^ P], axis=0)
            eds = np.sum((y[None, :] - (1.0 - 2.0 * cands)) ** 2, axis=1)
            order = np.argsort(eds, kind="stable")
            gaps.append(eds[order[1]] - eds[order[0]])
            j = int(np.argmin(eds[1:]))  # lowest pattern index among the best hops
            if eds[1 + j] < eds[0]:
                cen[k] = cands[1 + j]
                moved = True
            else:
                active[k] = False
        if not moved:
            break
    eds = [_ed(y, c) for c in cen]
    best = int(np.argmin(eds))
    for k, c in enumerate(cen):
        if not np.array_equal(c, cen[best]):
            gaps.append(eds[k] - eds[best])
    return min(gaps) if gaps else np.inf, cen[best]


def test_min_gap_against_brute_force_emulation(oracle_mod, rm26):
    """Seeded RM(2,6)+CRC-6 frames at 1 dB decoded in always-on mode: the
    oracle's min_gap and codeword equal the brute-force emulation from the same
    stage-1 anchors, frame by frame."""
    import synth

    _, P = rm26
    code = oracle_mod.rm_code(6, 2, crc_poly=0x21, crc_len=6)
    code = code.with_patterns(code.enumerate_codewords([16]))
    wl = synth.make_workload("rm26_crc6", 1.0, 40, seed=21)
    L, T = 4, 3
    out = code.decode(wl.y, L, T, aom=True, threads=2, want_anchors=True)
    for f in range(wl.B):
        y = wl.y[f].astype(np.float64)
        ul, _ = code.scl(y, L)
        anchors = [code.encode(u) for u in ul]
        gap, cw = _emulated_min_gap(y, anchors, P, T)
        assert oracle_mod.pack_bits(cw)[0] == out["cw"][f, 0], f
        assert out["min_gap"][f] == gap, (f, out["min_gap"][f], gap)
    # the gaps are not degenerate: most frames are far from the tie threshold
    thr = 1e-6 * np.sum(wl.y.astype(np.float64) ** 2, axis=1)
    assert np.mean(out["min_gap"] >= thr) > 0.5
