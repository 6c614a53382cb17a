"""Pins of the oracle's OSD(order) stage 1 (Sec. IV-A uses OSD anchors for the
RM code): each check uses something other than the oracle itself -- brute
force over the whole code, the ED identity, a GF(2) rank computation written
here, and frames whose answer is known by construction."""
import numpy as np
import pytest

import oracle
import synth


def _codebook(m, r):
    """All codewords of RM(r, m) in the Arikan form, by brute force over u."""
    F = oracle.kron_power(m)
    fz = oracle.rm_frozen(m, r)
    info = np.flatnonzero(fz == 0)
    k = info.size
    us = np.zeros((1 << k, F.shape[0]), np.int64)
    for a in range(1 << k):
        for t in range(k):
            if (a >> t) & 1:
                us[a, info[t]] = 1
    return (us @ F) % 2, F, fz


def _disc(y, cw):
    hd = (y < 0).astype(np.uint8)
    return float(np.sum(np.abs(y) * (cw != hd)))


def _is_codeword(cw, F, fz):
    u = (cw.astype(np.int64) @ F) % 2
    return not np.any(u[fz == 1])


@pytest.fixture(scope="module")
def rm15():
    return oracle.rm_code(5, 1)


def test_full_order_lists_the_whole_code_by_discrepancy(rm15):
    book, _, _ = _codebook(5, 1)
    rng = np.random.default_rng(1)
    for _ in range(20):
        y = synth.grid_quantize(rng.standard_normal(32) * 1.3).astype(np.float64)
        cl, d = rm15.osd(y, order=6, L=64)
        assert cl.shape[0] == 64
        # the same set of codewords as the code
        assert {bytes(c) for c in cl} == {bytes(c.astype(np.uint8)) for c in book}
        # ascending by the discrepancy computed here
        dd = np.array([_disc(y, c) for c in cl])
        assert np.array_equal(dd, d) and np.all(np.diff(dd) >= 0)
        # list[0] is the ML codeword
        ml, _ = rm15.ml(y)
        assert np.array_equal(cl[0], ml)


def test_discrepancy_orders_as_euclidean_distance():
    code = oracle.rm_code(6, 2)
    rng = np.random.default_rng(2)
    y = synth.grid_quantize(rng.standard_normal(64) * 1.2).astype(np.float64)
    cl, d = code.osd(y, order=2, L=32)
    for c, dq in zip(cl, d):
        ed = np.sum((y - (1.0 - 2.0 * c)) ** 2)
        assert ed == pytest.approx(np.sum(y ** 2) + 64 - 2 * np.sum(np.abs(y)) + 4 * dq, abs=1e-9)


def test_list_entries_are_distinct_codewords():
    code = oracle.rm_code(7, 2)
    F = oracle.kron_power(7)
    fz = oracle.rm_frozen(7, 2)
    rng = np.random.default_rng(3)
    for order in (0, 1, 2):
        y = synth.grid_quantize(rng.standard_normal(128) * 1.4).astype(np.float64)
        cl, d = code.osd(y, order=order, L=40)
        expect = 1 + (29 if order >= 1 else 0) + (29 * 28 // 2 if order >= 2 else 0)
        assert cl.shape[0] == min(40, expect)
        assert all(_is_codeword(c, F, fz) for c in cl)
        assert len({bytes(c) for c in cl}) == cl.shape[0]


def _mrb(y, G):
    """Most reliable basis by an independent greedy GF(2) rank walk."""
    order = sorted(range(y.size), key=lambda j: (-abs(y[j]), j))
    basis, chosen = [], []
    for j in order:
        col = G[:, j].copy()
        for b, piv in basis:
            if col[piv]:
                col ^= b
        nz = np.flatnonzero(col)
        if nz.size:
            basis.append((col, nz[0]))
            chosen.append(j)
        if len(chosen) == G.shape[0]:
            break
    return chosen


def test_order_zero_agrees_with_hard_decisions_on_the_most_reliable_basis():
    m, r = 5, 2
    book, F, fz = _codebook(m, r)
    code = oracle.rm_code(m, r)
    G = F[fz == 0].astype(np.uint8)
    rng = np.random.default_rng(4)
    for _ in range(10):
        y = synth.grid_quantize(rng.standard_normal(32) * 1.5).astype(np.float64)
        hd = (y < 0).astype(np.uint8)
        mrb = _mrb(y, G)
        assert len(mrb) == G.shape[0]
        cl, _ = code.osd(y, order=0, L=1)
        # the unique codeword that agrees with hd on the MRB, found in the whole code
        match = [c for c in book if np.array_equal(c[mrb], hd[mrb])]
        assert len(match) == 1 and np.array_equal(cl[0], match[0])


def test_two_strong_errors_in_the_basis_are_corrected_by_order_two():
    code = oracle.rm_code(6, 2)
    F = oracle.kron_power(6)
    fz = oracle.rm_frozen(6, 2)
    rng = np.random.default_rng(5)
    for _ in range(10):
        u = rng.integers(0, 2, 64) * (fz == 0)
        c = ((u @ F) % 2).astype(np.uint8)
        mag = 1.0 + np.arange(64)[rng.permutation(64)] / 128.0  # distinct reliabilities
        y = (1.0 - 2.0 * c) * mag
        top = np.argsort(-mag)[:6]
        flip = rng.choice(top, 2, replace=False)  # two errors among the most reliable positions
        y[flip] *= -1.0
        y = synth.grid_quantize(y).astype(np.float64)
        cl, _ = code.osd(y, order=2, L=4)
        assert np.array_equal(cl[0], c)
        cl1, _ = code.osd(y, order=1, L=4)
        assert not np.array_equal(cl1[0], c)  # one flip is not enough for two errors in the basis


@pytest.mark.parametrize("order", [1, 2])
def test_osd_stage_one_decode_never_beats_ml_and_keeps_its_best_anchor(order):
    patterns = oracle.rm_code(6, 2).enumerate_codewords([16])
    code = oracle.rm_code(6, 2, crc_poly=0x21, crc_len=6, patterns=patterns)
    wl = synth.make_workload("rm26_crc6", 1.0, 5, seed=9)  # brute-force ML is 2^22 codewords a frame
    out = code.decode(wl.y, 8, 4, osd_order=order, want_anchors=True, threads=2)
    F = oracle.kron_power(6)
    fz = oracle.rm_frozen(6, 2)
    for f in range(wl.y.shape[0]):
        y = wl.y[f].astype(np.float64)
        cw = oracle.unpack_bits(out["cw"][f], 64)
        assert _is_codeword(cw, F, fz)
        ml, ed_ml = code.ml(y)
        ed = np.sum((y - (1.0 - 2.0 * cw)) ** 2)
        assert ed >= ed_ml - 1e-9
        anchors = out["anchors"][f]
        cl, _ = code.osd(y, order=order, L=8)
        assert np.array_equal(anchors[:cl.shape[0]], cl)
        if out["flags"][f] & 1:  # stage 2 ran: the result is no worse than the best anchor
            ed_anchor = min(np.sum((y - (1.0 - 2.0 * a)) ** 2) for a in cl)
            assert ed <= ed_anchor + 1e-9


@pytest.mark.parametrize("order", [3, 4])
def test_high_order_lists_hold_every_candidate_once(order):
    """With L above the candidate count, OSD(order) returns sum_{i<=order}
    C(k, i) entries: c0 xor (rows of F) for distinct sets F of independent
    G_sys rows are distinct codewords. They come in ascending D, and every
    entry's D matches the discrepancy computed here."""
    import math

    code = oracle.rm_code(6, 2)
    F = oracle.kron_power(6)
    fz = oracle.rm_frozen(6, 2)
    k = int(np.sum(fz == 0))
    expect = sum(math.comb(k, i) for i in range(order + 1))
    rng = np.random.default_rng(20 + order)
    y = synth.grid_quantize(rng.standard_normal(64) * 1.3).astype(np.float64)
    cl, d = code.osd(y, order=order, L=expect + 5)
    assert cl.shape[0] == expect
    assert len({bytes(c) for c in cl}) == expect
    assert all(_is_codeword(c, F, fz) for c in cl[:: max(1, expect // 200)])
    assert np.all(np.diff(d) >= 0)
    pick = rng.choice(expect, 50, replace=False)
    assert np.array_equal(d[pick], np.array([_disc(y, cl[i]) for i in pick]))
