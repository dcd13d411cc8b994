"""Pins of the oracle's counts and local score (Eq. 3-4) and prior (Eq. 7-10)."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
LN10 = math.log(10.0)


def _rand_data(m, n, arity, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, int(a), size=m) for a in arity], axis=1).astype(np.uint8)


def _config_index(data, arity, parents):
    # mixed radix, first parent least significant (vectorised, independent of the C loop)
    idx = np.zeros(data.shape[0], np.int64)
    mult = 1
    for p in parents:
        idx += data[:, p].astype(np.int64) * mult
        mult *= int(arity[p])
    return idx, mult


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_counts_brute_force_and_invariants(seed):
    arity = np.array([2, 3, 4, 3, 2], np.uint8)
    data = _rand_data(257, 5, arity, seed)
    for child in range(5):
        others = [x for x in range(5) if x != child]
        for j in range(0, 4):
            for ps in [others[:j], others[-j:] if j else []]:
                c = oracle.counts(data, arity, child, ps)
                idx, q = _config_index(data, arity, ps)
                r = int(arity[child])
                brute = np.bincount(idx * r + data[:, child], minlength=q * r).reshape(q, r)
                assert np.array_equal(c, brute)
                assert c.sum() == data.shape[0]                       # sum = m
                if not ps:                                             # empty set = histogram
                    assert np.array_equal(c[0], np.bincount(data[:, child], minlength=r))
                # summing out the child gives the parents' own joint histogram
                assert np.array_equal(c.sum(axis=1), np.bincount(idx, minlength=q))


def test_k2_hand_worked_cases():
    g = json.load(open(os.path.join(GOLD, "k2_hand.json")))
    for case in g["cases"]:
        data = np.array(case["rows"], np.uint8)
        v = oracle.local_score(data, case["arity"], case["child"], case["parents"], kind=0)
        assert v == pytest.approx(case["log10"], rel=1e-14, abs=1e-15)


def _k2_exact_log10(cnt):
    """Closed form of Eq. (3) with alpha_ijk = 1 (K2):
    prod_c (r-1)! / (N_c + r - 1)! * prod_x N_cx!, as an exact rational."""
    q, r = cnt.shape
    num, den = 1, 1
    for c in range(q):
        Nc = int(cnt[c].sum())
        num *= math.factorial(r - 1)
        den *= math.factorial(Nc + r - 1)
        for x in range(r):
            num *= math.factorial(int(cnt[c, x]))
    f = Fraction(num, den)
    return math.log10(f.numerator) - math.log10(f.denominator)


@pytest.mark.parametrize("seed", [3, 4])
def test_k2_closed_form_exact_rationals(seed):
    arity = np.array([3, 2, 3, 4, 2, 3], np.uint8)
    data = _rand_data(180, 6, arity, seed)
    for child in range(6):
        others = [x for x in range(6) if x != child]
        for ps in ([], others[:1], others[1:3], others[2:5], others[:4]):
            cnt = oracle.counts(data, arity, child, ps)
            exact = _k2_exact_log10(cnt)
            v = oracle.local_score(data, arity, child, ps, kind=0)
            assert v == pytest.approx(exact, rel=1e-13, abs=1e-12)


def test_bdeu_against_scipy_gammaln():
    sp = pytest.importorskip("scipy.special")
    arity = np.array([3, 2, 4, 3], np.uint8)
    data = _rand_data(300, 4, arity, 11)
    for ess in (1.0, 10.0):
        for child in range(4):
            others = [x for x in range(4) if x != child]
            for ps in ([], others[:1], others[:2], others):
                cnt = oracle.counts(data, arity, child, ps).astype(np.float64)
                q, r = cnt.shape
                a_cx, a_c = ess / (q * r), ess / q
                ref = (np.sum(sp.gammaln(a_c) - sp.gammaln(a_c + cnt.sum(1)))
                       + np.sum(sp.gammaln(cnt + a_cx) - sp.gammaln(a_cx))) / LN10
                v = oracle.local_score(data, arity, child, ps, kind=1, ess=ess)
                assert v == pytest.approx(ref, rel=1e-12, abs=1e-11)


def test_bdeu_score_equivalence():
    # BDeu is score equivalent: a -> b and b -> a score the same
    arity = np.array([3, 2, 4], np.uint8)
    data = _rand_data(500, 3, arity, 5)
    for a, b in ((0, 1), (0, 2), (1, 2)):
        lhs = oracle.local_score(data, arity, a, [], 1, 7.0) + \
            oracle.local_score(data, arity, b, [a], 1, 7.0)
        rhs = oracle.local_score(data, arity, b, [], 1, 7.0) + \
            oracle.local_score(data, arity, a, [b], 1, 7.0)
        assert lhs == pytest.approx(rhs, rel=1e-12)
    # and the K2 score is not (guards against a kind mix-up)
    lhs = oracle.local_score(data, arity, 0, [], 0) + oracle.local_score(data, arity, 2, [0], 0)
    rhs = oracle.local_score(data, arity, 2, [], 0) + oracle.local_score(data, arity, 0, [2], 0)
    assert abs(lhs - rhs) > 1e-6


def test_no_data_gives_penalty_only():
    arity = np.array([2, 3, 4], np.uint8)
    data = np.zeros((0, 3), np.uint8)
    for kind in (0, 1):
        for ps in ([], [1], [1, 2]):
            v = oracle.local_score(data, arity, 0, ps, kind, 2.0, -1.0)
            assert v == len(ps) * -1.0


def test_structure_penalty_and_prior_fold():
    arity = np.array([2, 3, 2, 3], np.uint8)
    data = _rand_data(120, 4, arity, 9)
    R = np.array([[0.5, 1.0, 0.0, 0.75],
                  [0.25, 0.5, 0.5, 1.0],
                  [0.5, 0.5, 0.5, 0.5],
                  [0.0, 1.0, 0.9, 0.5]])
    for child in range(4):
        others = [x for x in range(4) if x != child]
        for ps in ([], others[:1], others[:2], others):
            base = oracle.local_score(data, arity, child, ps)
            pen = oracle.local_score(data, arity, child, ps, log10_gamma=-0.7)
            assert pen - base == pytest.approx(-0.7 * len(ps), abs=1e-12)
            pri = oracle.local_score(data, arity, child, ps, R=R)
            ppf = sum(100.0 * (R[child, p] - 0.5) ** 3 for p in ps)
            assert pri - base == pytest.approx(ppf, abs=1e-12)


def test_ppf_closed_form_and_requirements():
    # Eq. (10) at the grid points, and the sign requirements of Sec. IV
    for r, v in ((0.0, -12.5), (0.25, -1.5625), (0.5, 0.0), (0.75, 1.5625), (1.0, 12.5)):
        assert oracle.ppf(r) == v
    for r in np.linspace(0, 1, 101):
        p = oracle.ppf(float(r))
        assert (p > 0) == (r > 0.5) and (p < 0) == (r < 0.5)
        assert oracle.ppf(1.0 - float(r)) == pytest.approx(-p, abs=1e-12)


def test_state_relabelling_gives_identical_bits():
    # permuting the states of a parent permutes the count table's rows; the canonical
    # summation order makes the two scores bit-identical (ties stay exact ties)
    arity = np.array([3, 3, 2], np.uint8)
    data = _rand_data(400, 3, arity, 21)
    d2 = data.copy()
    perm = np.array([2, 0, 1], np.uint8)
    d2[:, 1] = perm[data[:, 1]]
    for kind in (0, 1):
        a = oracle.local_score(data, arity, 0, [1, 2], kind, 3.0)
        b = oracle.local_score(d2, arity, 0, [1, 2], kind, 3.0)
        assert a == b


def test_table_layout_matches_local_score():
    data, arity, k, R, _ = synth.workload("n6_k2_m100")
    T = oracle.build_table(data, arity, k)
    n = data.shape[1]
    S = oracle.num_sets(n - 1, k)
    assert T.shape == (n, S)
    for i in range(n):
        for r in range(S):
            ps = oracle.parent_set(n, k, i, r)
            assert T[i, r] == oracle.local_score(data, arity, i, ps)
