"""The integer arithmetic and the sorting network of the stage-1 SC-list
kernel, checked on the CPU as rules (no GPU code involved).

* The min-sum f of the kernel, max(min(a,b), -max(a,b)), equals
  sign(a) sign(b) min(|a|,|b|) with sign(0) = +1 (the form the oracle's
  Sec. III-A recursion uses), and with P(x) = max(0, -x) the identity
  P(f(a,b)) + P(a+b) = P(a) + P(b) holds, which lets an all-frozen node add
  sum_k P(input_k) in one step.
* The bitonic network of the list step, with each lane's stage directions
  taken from a bit mask computed once per lane, sorts every input of every
  segment width (0-1 principle), and the merge keeps the LW smallest of two
  ascending sequences in ascending order.
* The 32-bit keys (metric relative to the list's lower bound, parent lane,
  bit) order the children exactly as (metric, parent position, bit) while
  the relative metric is below 2^25, and an empty lane's key sorts last.
* The bound behind the 32-bit sum of an all-frozen node: every input of a
  node of size S is at most 2^23 n / S in magnitude, so S inputs sum to at
  most 2^23 n <= 2^30 for n <= 128."""
import itertools

import numpy as np
import pytest


def f_kernel(a, b):
    return np.maximum(np.minimum(a, b), -np.maximum(a, b))


def f_sign_magnitude(a, b):
    m = np.minimum(np.abs(a), np.abs(b))
    return np.where((a ^ b) < 0, -m, m)


def P(x):
    return np.maximum(0, -x)


def test_minsum_f_equals_sign_magnitude_form():
    r = np.arange(-64, 65, dtype=np.int64)
    a, b = np.meshgrid(r, r)
    assert np.array_equal(f_kernel(a, b), f_sign_magnitude(a, b))
    rng = np.random.default_rng(1)
    big = 1 << 30
    a = rng.integers(-big, big + 1, 200000)
    b = rng.integers(-big, big + 1, 200000)
    assert np.array_equal(f_kernel(a, b), f_sign_magnitude(a, b))
    # the signs of zero: f(0, b) = 0 and f(a, 0) = 0
    assert np.all(f_kernel(np.zeros_like(a), b) == 0) and np.all(f_kernel(a, np.zeros_like(b)) == 0)


def test_frozen_node_increment_identity():
    r = np.arange(-40, 41, dtype=np.int64)
    a, b = np.meshgrid(r, r)
    assert np.array_equal(P(f_kernel(a, b)) + P(a + b), P(a) + P(b))


def _frozen_sum_leaf_by_leaf(x):
    """Metric increment of an all-frozen node decided leaf by leaf (every u = 0):
    f on the left half, recurse, g = b + a (left codeword 0) on the right half."""
    if x.shape[0] == 1:
        return int(P(x[0]))
    h = x.shape[0] // 2
    a, b = x[:h], x[h:]
    return _frozen_sum_leaf_by_leaf(f_kernel(a, b)) + _frozen_sum_leaf_by_leaf(b + a)


@pytest.mark.parametrize("S", [2, 4, 8, 16, 32])
def test_frozen_node_one_step_sum(S):
    rng = np.random.default_rng(S)
    for _ in range(50):
        x = rng.integers(-1000, 1001, S).astype(np.int64)
        assert _frozen_sum_leaf_by_leaf(x) == int(P(x).sum())


def test_frozen_node_sum_fits_int32():
    grid_max = (1 << 23) - 1
    for n in (32, 64, 128):
        for S in [1 << i for i in range(1, n.bit_length() - 1)]:  # S < n
            per_input = grid_max * (n // S)  # g sums double the magnitude per level
            assert S * per_input <= (1 << 30) < (1 << 31) - 1


def sort_dirs(lane, LW):
    d, s = 0, 0
    k = 2
    while k <= LW:
        j = k >> 1
        while j > 0:
            if ((lane & k) == 0) == ((lane & j) == 0):
                d |= 1 << s
            s += 1
            j >>= 1
        k <<= 1
    return d


def seg_sort(x, LW):
    """The kernel's network on one segment: x[lane] is lane's key."""
    x = list(x)
    dirs = [sort_dirs(l, LW) for l in range(LW)]
    s = 0
    k = 2
    while k <= LW:
        j = k >> 1
        while j > 0:
            o = [x[l ^ j] for l in range(LW)]
            x = [min(x[l], o[l]) if dirs[l] >> s & 1 else max(x[l], o[l]) for l in range(LW)]
            s += 1
            j >>= 1
        k <<= 1
    return x


def seg_merge_low(a, b, LW):
    x = [min(a[l], b[LW - 1 - l]) for l in range(LW)]
    j = LW // 2
    while j > 0:
        o = [x[l ^ j] for l in range(LW)]
        x = [max(x[l], o[l]) if l & j else min(x[l], o[l]) for l in range(LW)]
        j >>= 1
    return x


@pytest.mark.parametrize("LW", [2, 4, 8, 16])
def test_network_sorts_every_binary_input(LW):
    for bits in itertools.product((0, 1), repeat=LW):
        assert seg_sort(bits, LW) == sorted(bits), bits


def test_network_sorts_random_keys_32():
    rng = np.random.default_rng(32)
    for _ in range(300):
        x = rng.integers(0, 50, 32).tolist()
        assert seg_sort(x, 32) == sorted(x)


@pytest.mark.parametrize("LW", [2, 4, 8, 16, 32])
def test_merge_keeps_the_smallest(LW):
    rng = np.random.default_rng(LW)
    for _ in range(200):
        a = sorted(rng.integers(0, 3 * LW, LW).tolist())
        b = sorted(rng.integers(0, 3 * LW, LW).tolist())
        assert seg_merge_low(a, b, LW) == sorted(a + b)[:LW]


def test_relative_keys_order_children_as_metric_parent_bit():
    rng = np.random.default_rng(5)
    LW = 8
    for trial in range(300):
        count = int(rng.integers(1, LW + 1))
        spread = 1 << int(rng.integers(1, 24))
        pref = int(rng.integers(0, 1 << 40))
        pm = pref + rng.integers(0, spread, count)
        lam = rng.integers(-spread, spread + 1, count)
        children = []  # (metric, parent, bit)
        keys = []
        for l in range(LW):
            if l < count:
                hd = 1 if lam[l] < 0 else 0
                a = abs(int(lam[l]))
                d0 = int(pm[l]) - pref
                assert d0 + a < (1 << 25)
                children += [(int(pm[l]), l, hd), (int(pm[l]) + a, l, hd ^ 1)]
                keys += [(d0 << 6) | (l << 1) | hd, ((d0 + a) << 6) | (l << 1) | (hd ^ 1)]
            else:
                keys += [0xFFFFFFFF, 0xFFFFFFFF]
        assert max(k for k in keys if k != 0xFFFFFFFF) < 1 << 31
        got = [(pref + (k >> 6), (k >> 1) & 31, k & 1) for k in sorted(keys)[:2 * count]]
        assert got == sorted(children), trial
