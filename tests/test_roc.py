"""Host-side accuracy bookkeeping (the ROC study): rates on hand-made graphs, the prior
schedule's assignments and seeding, and the noise injection's flip rate."""
import numpy as np

import synth
from paper_1210_5128_gb300 import roc


def test_rates_on_a_hand_example():
    # true: 0 -> 1, 1 -> 2 ; learned: 0 -> 1 (right), 2 -> 1 (reversed 1 -> 2), 0 -> 2 (extra)
    T = np.zeros((3, 3), np.uint8)
    T[1, 0] = 1
    T[2, 1] = 1
    L = np.zeros((3, 3), np.uint8)
    L[1, 0] = 1
    L[1, 2] = 1
    L[2, 0] = 1
    tp, fp = roc.tp_fp(L, T)
    assert tp == 0.5                       # 1 of 2 directed edges
    assert fp == 2 / 4                     # 2 of the 4 directed non-edges
    tp_s, fp_s = roc.tp_fp(L, T, skeleton=True)
    assert tp_s == 1.0                     # both adjacencies found
    assert fp_s == 1.0                     # the one non-adjacent pair {0, 2} was added
    assert roc.tp_fp(T, T) == (1.0, 0.0)
    assert roc.tp_fp(np.zeros_like(T), T) == (0.0, 0.0)


def test_true_adjacency_matches_parents():
    net = synth.random_network(12, 3, 2, 5)
    A = roc.true_adjacency(net)
    for i in range(12):
        assert sorted(np.nonzero(A[i])[0].tolist()) == list(net.parents[i])


def test_prior_schedule():
    n = 30
    rng = np.random.default_rng(1)
    T = (rng.random((n, n)) < 0.1).astype(np.uint8)
    L = (rng.random((n, n)) < 0.1).astype(np.uint8)
    np.fill_diagonal(T, 0)
    np.fill_diagonal(L, 0)
    R = roc.prior_from_errors(L, T, 0.8, 0.1, 1.0, seed=3)
    missed = (T == 1) & (L == 0)
    added = (T == 0) & (L == 1)
    assert (R[missed] == 0.8).all() and (R[added] == 0.1).all()
    assert (R[~missed & ~added] == 0.5).all()
    R0 = roc.prior_from_errors(L, T, 0.8, 0.1, 0.0, seed=3)
    assert (R0 == 0.5).all()
    Ra = roc.prior_from_errors(L, T, 0.7, 0.2, 0.4, seed=9)
    Rb = roc.prior_from_errors(L, T, 0.7, 0.2, 0.4, seed=9)
    assert np.array_equal(Ra, Rb)
    frac = ((Ra != 0.5) & (missed | added)).sum() / (missed | added).sum()
    assert 0.2 < frac < 0.6


def test_flip_noise_rate_and_binary():
    d = np.zeros((4000, 20), np.uint8)
    f = roc.flip_noise(d, 0.1, 4)
    assert set(np.unique(f)) <= {0, 1}
    assert abs(f.mean() - 0.1) < 0.01
    assert np.array_equal(roc.flip_noise(d, 0.0, 4), d)
    assert np.array_equal(roc.flip_noise(1 - d, 1.0, 4), d)
