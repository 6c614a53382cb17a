"""Pins for the oracle's stage-1 SC-list decoder (Sec. III-A, min-sum reading).

The oracle computes each leaf LLR from scratch with explicit re-encoding
matrices. The reference here is written differently: the classic recursive
successive-cancellation decoder in which every node returns the codeword of
its sub-block, so a wrong f, g, sign rule, index split or encoder in the
oracle shows up as a disagreement."""
import math

import numpy as np
import pytest


def _f(a, b):
    sa = 1.0 if a >= 0 else -1.0
    sb = 1.0 if b >= 0 else -1.0
    return sa * sb * min(abs(a), abs(b))


def sc_ref(lam, frozen, forced=None):
    """Recursive SC decoding: returns (u, c, pm). With ``forced`` the info
    decisions are imposed and pm is the min-sum path metric of that u."""
    n = len(lam)
    if n == 1:
        hd = 0 if lam[0] >= 0 else 1
        if frozen[0]:
            u = 0
        elif forced is not None:
            u = int(forced[0])
        else:
            u = hd
        return [u], [u], (abs(lam[0]) if u != hd else 0.0)
    h = n // 2
    a, b = lam[:h], lam[h:]
    uL, cL, pmL = sc_ref([_f(x, y) for x, y in zip(a, b)], frozen[:h], None if forced is None else forced[:h])
    right = [y + (1 - 2 * c) * x for x, y, c in zip(a, b, cL)]
    uR, cR, pmR = sc_ref(right, frozen[h:], None if forced is None else forced[h:])
    return uL + uR, [p ^ q for p, q in zip(cL, cR)] + cR, pmL + pmR


def _noisy_frames(oracle_mod, code, B, sigma, seed):
    rng = np.random.default_rng(seed)
    info = np.flatnonzero(code.frozen == 0)
    ys, cs = [], []
    for _ in range(B):
        u = np.zeros(code.n, np.uint8)
        u[info] = rng.integers(0, 2, info.size)
        c = code.encode(u)
        y = (1.0 - 2.0 * c) + sigma * rng.standard_normal(code.n)
        y = np.rint(y * 2 ** 19) / 2 ** 19
        ys.append(y)
        cs.append(c)
    return np.array(ys), np.array(cs)


@pytest.mark.parametrize("m,r", [(5, 1), (6, 2), (7, 2), (4, 2)])
def test_sc_list1_equals_recursive_sc(oracle_mod, m, r):
    code = oracle_mod.rm_code(m, r)
    ys, _ = _noisy_frames(oracle_mod, code, 40, 1.1, seed=m * 10 + r)
    for y in ys:
        ul, pm = code.scl(y, 1)
        u, c, pmr = sc_ref(list(y), list(code.frozen))
        assert ul.shape[0] == 1
        assert ul[0].tolist() == u
        assert code.encode(ul[0]).tolist() == c
        assert pm[0] == pmr


def test_sc_random_frozen_sets(oracle_mod):
    rng = np.random.default_rng(3)
    for trial in range(20):
        n = 32
        fz = (rng.random(n) < 0.6).astype(np.uint8)
        code = oracle_mod.Code(n, fz, int((fz == 0).sum()))
        y = np.rint(rng.standard_normal(n) * 2 ** 19) / 2 ** 19
        ul, pm = code.scl(y, 1)
        u, c, pmr = sc_ref(list(y), list(fz))
        assert ul[0].tolist() == u and pm[0] == pmr


def test_full_list_is_codebook_with_bruteforce_metrics(oracle_mod):
    """With L = 2^k nothing is pruned: the list is the whole code and every
    entry carries the min-sum metric of its u, evaluated independently."""
    code = oracle_mod.rm_code(5, 1)  # k = 6
    ys, _ = _noisy_frames(oracle_mod, code, 6, 1.0, seed=11)
    info = np.flatnonzero(code.frozen == 0)
    for y in ys:
        ul, pm = code.scl(y, 64)
        assert ul.shape[0] == 64
        got = {tuple(u): p for u, p in zip(ul.tolist(), pm.tolist())}
        assert len(got) == 64
        for a in range(64):
            u = np.zeros(32, np.uint8)
            u[info] = [(a >> t) & 1 for t in range(6)]
            _, _, pmr = sc_ref(list(y), list(code.frozen), forced=list(u))
            assert got[tuple(u.tolist())] == pmr
        assert np.all(np.diff(pm) >= 0)


def test_list_sorted_distinct_and_frozen_zero(oracle_mod):
    code = oracle_mod.rm_code(6, 2)
    ys, _ = _noisy_frames(oracle_mod, code, 20, 1.2, seed=5)
    for y in ys:
        for L in (2, 4, 8, 16, 32):
            ul, pm = code.scl(y, L)
            assert ul.shape[0] == L
            assert np.all(np.diff(pm) >= 0)
            assert len({tuple(u) for u in ul.tolist()}) == L
            # frozen positions are zero in every path
            assert not ul[:, code.frozen.astype(bool)].any()


def leaf_llrs_ref(lam, u):
    """Recursive SC with every decision imposed by u: (codeword of the block,
    LLR seen at each leaf). Written like ``sc_ref``, independently of the oracle."""
    if len(lam) == 1:
        return [int(u[0])], [lam[0]]
    h = len(lam) // 2
    a, b = lam[:h], lam[h:]
    cL, lL = leaf_llrs_ref([_f(x, y) for x, y in zip(a, b)], u[:h])
    cR, lR = leaf_llrs_ref([y + (1 - 2 * c) * x for x, y, c in zip(a, b, cL)], u[h:])
    return [p ^ q for p, q in zip(cL, cR)] + cR, lL + lR


def scl_breadth_first_ref(lam, frozen, L):
    """SC-list by its definition: every surviving path is extended leaf by
    leaf; at an information leaf each path spawns both bits, the metric grows
    by |lambda| when the bit disagrees with the hard decision, and the L best
    children are kept in the order (metric, parent position, bit); a frozen leaf
    takes 0 and keeps the order; the final list is stably sorted by metric.
    Each leaf LLR comes from a fresh recursive SC pass over the path's prefix."""
    n = len(lam)
    paths = [([], 0.0)]
    for i in range(n):
        children = []
        for q, (u, pm) in enumerate(paths):
            li = leaf_llrs_ref(lam, u + [0] * (n - len(u)))[1][i]
            hd = 0 if li >= 0 else 1
            for bit in ((0,) if frozen[i] else (0, 1)):
                children.append((u + [bit], pm + (abs(li) if bit != hd else 0.0), q, bit))
        if not frozen[i]:
            children.sort(key=lambda t: (t[1], t[2], t[3]))
            children = children[:L]
        paths = [(t[0], t[1]) for t in children]
    paths.sort(key=lambda t: t[1])
    return paths


@pytest.mark.parametrize("m,r,Ls,frames", [(5, 1, (2, 3, 8, 32), 8), (6, 2, (2, 4, 8, 16), 5), (7, 2, (16,), 2)])
def test_list_equals_breadth_first_reference(oracle_mod, m, r, Ls, frames):
    """1 < L < 2^k, where pruning decides what survives: the oracle's list
    (paths and metrics, in order) equals the breadth-first reference."""
    code = oracle_mod.rm_code(m, r)
    ys, _ = _noisy_frames(oracle_mod, code, frames, 1.3, seed=40 + m)
    for y in ys:
        for L in Ls:
            ul, pm = code.scl(y, L)
            want = scl_breadth_first_ref(list(y), list(code.frozen), L)
            assert [list(u) for u in ul.tolist()] == [p[0] for p in want], (m, L)
            assert pm.tolist() == [p[1] for p in want], (m, L)


def test_noiseless_frame_decodes_with_zero_metric(oracle_mod):
    code = oracle_mod.rm_code(6, 2)
    ys, cs = _noisy_frames(oracle_mod, code, 10, 0.0, seed=9)
    for y, c in zip(ys, cs):
        ul, pm = code.scl(y, 8)
        assert code.encode(ul[0]).tolist() == c.tolist()
        assert pm[0] == 0.0 and pm[1] > 0


def test_all_zero_llr_tie_rule(oracle_mod):
    """Every LLR is 0, so every metric ties: the order is (parent position, u).
    Then list[q] carries the binary expansion of q (first decided bit as the
    most significant) in the last log2(L) info positions and zeros elsewhere."""
    code = oracle_mod.rm_code(6, 2)
    info = np.flatnonzero(code.frozen == 0)
    for L in (1, 2, 8, 32):
        ul, pm = code.scl(np.zeros(64), L)
        assert np.all(pm == 0)
        b = int(math.log2(L))
        for q in range(L):
            want = np.zeros(64, np.uint8)
            for t in range(b):
                want[info[info.size - b + t]] = (q >> (b - 1 - t)) & 1
            assert ul[q].tolist() == want.tolist()
