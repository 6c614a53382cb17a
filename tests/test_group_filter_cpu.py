"""The candidate-group filter of the tensor-core scoring path, checked on the
CPU as a rule (no GPU code involved).

The scoring kernel keeps, per row, the groups of 8 consecutive patterns whose
smallest approximate score lies within 2 eps of the row's smallest one (at
most four; a fourth one inside the band sends the row to a full rescan), and
the resolution scores every pattern of those groups exactly and takes the
smallest exact score, lowest index on ties. The claim is that this equals
Algorithm 1's argmin of the exact scores whenever every approximate score is
within eps of its exact one, and that a row whose smallest approximate score
exceeds eps has no pattern of negative exact score. Checked here with the
oracle's exact gains (Eq. (5)) of RM(2,6) rows, approximate scores perturbed
adversarially inside the eps bound, and integer scores with many exact ties."""
import numpy as np
import pytest

G, K = 8, 4


def group_filter(approx, eps):
    """Groups kept by the filter (ascending by group minimum, lower group
    first on equal minima) and whether the list is full inside the band."""
    P = approx.shape[0]
    ng = (P + G - 1) // G
    gmin = np.array([approx[g * G:(g + 1) * G].min() for g in range(ng)])
    order = np.argsort(gmin, kind="stable")
    band = [int(g) for g in order if gmin[g] <= gmin[order[0]] + 2 * eps]
    return band[:K], len(band) >= K


def resolve(exact, kept):
    best, bp = None, None
    for g in kept:
        for p in range(g * G, min((g + 1) * G, exact.shape[0])):
            if best is None or exact[p] < best or (exact[p] == best and p < bp):
                best, bp = exact[p], p
    return bp


def exact_argmin(exact):
    return int(np.flatnonzero(exact == exact.min())[0])


@pytest.fixture(scope="module")
def rm26(oracle_mod):
    code = oracle_mod.rm_code(6, 2)
    return code.with_patterns(code.enumerate_codewords([16]))


def _check(exact, approx, eps):
    kept, full = group_filter(approx, eps)
    if not full:
        assert resolve(exact, kept) == exact_argmin(exact)
    # the stop rule: no pattern can improve when even the smallest approximate score exceeds eps
    if approx.min() > eps:
        assert exact.min() > 0.0
    return full


def test_resolution_equals_the_exact_argmin_on_rm26_rows(rm26, oracle_mod):
    rng = np.random.default_rng(11)
    P = rm26.patterns.shape[0]
    pats = oracle_mod.unpack_bits(rm26.patterns, 64)
    fulls = 0
    for trial in range(300):
        y = np.round((rng.standard_normal(64) * 1.2 + 0.3) * 2 ** 19) / 2 ** 19
        c = np.zeros(64, np.uint8)
        for p in rng.integers(0, P, 3):
            c ^= pats[p]
        exact = -rm26.gains(y, c) / 2.0
        eps = 2.0 ** -14 * np.abs(y).sum()
        # adversarial perturbation inside the bound: the exact argmin pushed up by
        # eps, its nearest rivals pushed down by eps, the rest at random
        noise = rng.uniform(-eps, eps, P)
        a = exact_argmin(exact)
        noise[a] = eps
        for q in np.argsort(exact)[1:6]:
            noise[q] = -eps
        fulls += _check(exact, exact + noise, eps)
    assert fulls < 300  # the rule is exercised, not just the rescan


def test_resolution_with_exact_ties_keeps_the_lowest_index():
    rng = np.random.default_rng(12)
    for trial in range(500):
        P = int(rng.integers(1, 200))
        exact = rng.integers(-3, 4, P).astype(np.float64)  # many exact ties
        eps = 0.25
        approx = exact + rng.uniform(-eps, eps, P)
        _check(exact, approx, eps)


def test_partial_last_group_and_single_pattern():
    exact = np.array([3.0, 2.0, 5.0, 1.0, 4.0, 9.0, 7.0, 8.0, 0.5, 6.0])  # 2 groups, the second partial
    assert resolve(exact, group_filter(exact, 1e-3)[0]) == 8
    assert resolve(np.array([-1.0]), group_filter(np.array([-1.0]), 0.0)[0]) == 0


def test_full_band_is_reported():
    exact = np.zeros(64)  # every pattern ties: all eight groups sit in the band
    kept, full = group_filter(exact, 0.0)
    assert full and kept == [0, 1, 2, 3]
