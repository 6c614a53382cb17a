"""Pins for the oracle's code algebra (Sec. II-B, II-C): the Arikan kernel
power, the Reed-Muller frozen sets, the CRC, the codeword enumeration that
builds S_r(0), and the weight distributions -- each checked against facts
fixed by mathematics or printed in the paper, not against the oracle itself."""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_kron_power_is_submask_rule_and_involution(oracle_mod):
    for m in range(1, 8):
        F = oracle_mod.kron_power(m)
        n = 1 << m
        for i in range(n):
            for j in range(n):
                assert F[i, j] == (1 if (i & j) == j else 0)
        # F is its own inverse over F2 ([[1,0],[1,1]]^2 = I mod 2)
        assert np.array_equal((F.astype(np.int64) @ F.astype(np.int64)) % 2, np.eye(n, dtype=np.int64))
        # row i has weight 2^popcount(i)
        assert all(F[i].sum() == 2 ** bin(i).count("1") for i in range(n))


@pytest.mark.parametrize("m,r,k", [(5, 1, 6), (6, 2, 22), (7, 2, 29), (5, 0, 1), (4, 4, 16)])
def test_rm_dimension(oracle_mod, m, r, k):
    # dim RM(r, m) = sum_{i<=r} C(m, i)
    assert k == sum(math.comb(m, i) for i in range(r + 1))
    assert int((oracle_mod.rm_frozen(m, r) == 0).sum()) == k


def test_crc_hand_worked_examples(oracle_mod):
    """g(x) = x^6 + x^5 + 1. x^6 = x^5 + 1 (mod g), so a message whose only
    one is its last bit (m(x) = 1) has remainder x^5 + 1 -> bits 100001; for
    m(x) = x: x^7 = x^6 + x = x^5 + x + 1 -> 100011; for m(x) = x^2:
    x^8 = x^6 + x^2 + x = x^5 + x^2 + x + 1 -> 100111."""
    with open(os.path.join(GOLDEN, "crc6_hand_examples.json")) as fh:
        gold = json.load(fh)
    for case in gold["cases"]:
        msg = np.array(case["msg"], np.uint8)
        r = oracle_mod.crc(msg, int(gold["poly"], 16), gold["len"])
        assert r.tolist() == case["crc"], case


def test_crc_linear_zero_and_self_check(oracle_mod):
    rng = np.random.default_rng(5)
    for _ in range(200):
        a = rng.integers(0, 2, 16).astype(np.uint8)
        b = rng.integers(0, 2, 16).astype(np.uint8)
        ra, rb = oracle_mod.crc(a, 0x21, 6), oracle_mod.crc(b, 0x21, 6)
        assert np.array_equal(oracle_mod.crc(a ^ b, 0x21, 6), ra ^ rb)
        # appending the remainder makes the whole word divisible by g(x)
        assert not oracle_mod.crc(np.concatenate([a, ra]), 0x21, 6).any()
    assert not oracle_mod.crc(np.zeros(16, np.uint8), 0x21, 6).any()
    # CRC-11 of Sec. IV-A, g = 1 + x^5 + x^9 + x^10 + x^11 -> 0x621: same properties
    a = rng.integers(0, 2, 16).astype(np.uint8)
    assert not oracle_mod.crc(np.concatenate([a, oracle_mod.crc(a, 0x621, 11)]), 0x621, 11).any()


def _min_weight_count(r, m):
    """A_{2^(m-r)} of RM(r, m) = 2^r prod_{i=0}^{m-r-1} (2^(m-i) - 1)/(2^(m-r-i) - 1)."""
    v = Fraction(2 ** r)
    for i in range(m - r):
        v *= Fraction(2 ** (m - i) - 1, 2 ** (m - r - i) - 1)
    assert v.denominator == 1
    return int(v)


def test_min_weight_closed_forms():
    assert _min_weight_count(1, 5) == 62
    assert _min_weight_count(2, 6) == 2604
    assert _min_weight_count(2, 7) == 10668


def _krawtchouk(n, k, x):
    return sum((-1) ** j * math.comb(x, j) * math.comb(n - x, k - j) for j in range(k + 1))


def _check_distribution(A, n, k, dual_d):
    A = [int(a) for a in A]
    assert A[0] == 1 and sum(A) == 2 ** k
    assert all(A[w] == A[n - w] for w in range(n + 1))  # all-ones word is in the code
    # MacWilliams: B_j = 2^-k sum_w A_w K_j(w) is the dual's distribution
    B = [Fraction(sum(A[w] * _krawtchouk(n, j, w) for w in range(n + 1)), 2 ** k) for j in range(n + 1)]
    assert all(b.denominator == 1 and b >= 0 for b in B)
    assert B[0] == 1 and sum(B) == 2 ** (n - k)
    assert all(B[j] == 0 for j in range(1, dual_d)) and B[dual_d] > 0


def test_weight_distribution_rm15(oracle_mod):
    code = oracle_mod.rm_code(5, 1)
    A = code.weight_distribution()
    assert {w: int(a) for w, a in enumerate(A) if a} == {0: 1, 16: 62, 32: 1}
    _check_distribution(A, 32, 6, dual_d=4)  # dual of RM(1,5) is RM(3,5), d = 4


def test_weight_distribution_rm26(oracle_mod):
    code = oracle_mod.rm_code(6, 2)
    A = code.weight_distribution()
    assert A[16] == _min_weight_count(2, 6)
    assert all(A[w] == 0 for w in range(1, 16))
    _check_distribution(A, 64, 22, dual_d=8)  # dual of RM(2,6) is RM(3,6), d = 8


def _flats(m, d):
    """Incidence vectors (as ints, bit j = point j) of all d-dimensional affine
    subspaces of F2^m: the minimum-weight codewords of RM(m-d, m)."""
    subspaces = set()
    for piv in itertools.combinations(range(m), d):
        # reduced row-echelon bases with pivots at piv; free entries at non-pivot
        # columns to the right of each pivot
        free = [[c for c in range(piv[i] + 1, m) if c not in piv] for i in range(d)]
        for bits in itertools.product(*[itertools.product((0, 1), repeat=len(f)) for f in free]):
            rows = []
            for i in range(d):
                v = 1 << piv[i]
                for c, b in zip(free[i], bits[i]):
                    if b:
                        v |= 1 << c
                rows.append(v)
            span = {0}
            for rv in rows:
                span |= {s ^ rv for s in span}
            subspaces.add(frozenset(span))
    vecs = set()
    for V in subspaces:
        for a in range(1 << m):
            vecs.add(sum(1 << (a ^ v) for v in V))
    return vecs


def _as_ints(words):
    return {sum(int(w) << (64 * q) for q, w in enumerate(row)) for row in words}


@pytest.mark.parametrize("m,r", [(5, 1), (6, 2)])
def test_min_weight_set_equals_flats(oracle_mod, m, r):
    code = oracle_mod.rm_code(m, r)
    d = 2 ** (m - r)
    pats = code.enumerate_codewords([d])
    got = _as_ints(pats)
    assert len(got) == len(pats) == _min_weight_count(r, m)
    assert got == _flats(m, m - r)


def test_min_weight_set_rm27_equals_flats(oracle_mod):
    code = oracle_mod.rm_code(7, 2)
    pats = code.enumerate_codewords([32])
    assert len(pats) == 10668
    assert _as_ints(pats) == _flats(7, 5)


def test_table2_sphere_size_reading():
    """Table II prints |S_1(0)| = 10,688 for RM(128,29); the closed form gives
    10,668 weight-32 codewords. The fixture records the printed value and the
    reading taken (a typo in the table)."""
    with open(os.path.join(GOLDEN, "table2_sphere_sizes.json")) as fh:
        gold = json.load(fh)
    rm = gold["rm_128_29"]
    assert rm["printed"] == 10688
    assert rm["reading"] == _min_weight_count(2, 7) == 10668


def test_enumeration_order_and_codeword_property(oracle_mod):
    code = oracle_mod.rm_code(6, 2)
    pats = code.enumerate_codewords([16, 24])
    assert len(pats) == 2604 + 291648
    F = oracle_mod.kron_power(6).astype(np.int64)
    bits = oracle_mod.unpack_bits(pats[::997], 64).astype(np.int64)
    u = (bits @ F) % 2
    assert not u[:, code.frozen.astype(bool)].any()  # H c = 0: u is zero on frozen indices
    w = bits.sum(axis=1)
    assert set(w.tolist()) <= {16, 24}
    # canonical order: weight ascending, then message integer (lowest info index = MSB)
    info = np.flatnonzero(code.frozen == 0)
    allbits = oracle_mod.unpack_bits(pats, 64).astype(np.int64)
    uu = (allbits @ F) % 2
    msgint = np.zeros(len(pats), np.int64)
    for t, i in enumerate(info):
        msgint |= uu[:, i] << (len(info) - 1 - t)
    wts = allbits.sum(axis=1)
    key = wts * (1 << 40) + msgint
    assert np.all(np.diff(key) > 0)
