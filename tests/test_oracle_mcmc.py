"""Pins of the oracle's sampler (Sec. III.C): RNG, exact stationary law, edge
frequencies, best graph, and the ESS estimator."""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth


def test_philox4x64_matches_numpy():
    """numpy's Philox bit generator is Philox4x64-10; it increments the counter before
    each block, so its first block is Philox(counter + 1)."""
    for key, ctr in [((0, 0), (0, 0, 0, 0)), ((123, 456), (7, 8, 9, 10)),
                     ((2**64 - 1, 2**63), (2**64 - 1, 5, 6, 2**64 - 2)),
                     ((0xB4E50003, 0), (41, 3, 0, 0))]:
        g = np.random.Philox(key=np.array(key, np.uint64), counter=np.array(ctr, np.uint64))
        ref = g.random_raw(8)
        c = list(ctr)
        for blk in range(2):
            c[0] = (c[0] + 1) % 2**64
            if c[0] == 0:
                c[1] = (c[1] + 1) % 2**64
            assert list(oracle.philox4x64(c, key)) == list(ref[4 * blk:4 * blk + 4])


def test_init_order_and_pair_decode():
    for n in (2, 6, 20, 60):
        for c in range(5):
            o = oracle.init_order(99, c, n)
            assert sorted(o.tolist()) == list(range(n))
        P = n * (n - 1) // 2
        seen = [oracle.pair_decode(n, i) for i in range(P)]
        assert seen == list(itertools.combinations(range(n), 2))


def _small_problem(n=4, m=25, seed=0):
    net = synth.random_network(n, 2, 2, 1234 + seed)
    data = synth.forward_sample(net, m, 99 + seed)
    arity = net.arity
    k = 2
    return oracle.build_table(data, arity, k), k


def _exact(T, k, temper=1.0):
    n = T.shape[0]
    orders = [np.array(o, np.uint8) for o in itertools.permutations(range(n))]
    sc = np.array([oracle.order_score(T, k, o)[0] for o in orders])
    w = np.power(10.0, temper * (sc - sc.max()))
    pi = w / w.sum()
    edge = np.zeros((n, n))
    for o, p in zip(orders, pi):
        _, br = oracle.order_score(T, k, o)
        edge += p * oracle.greedy_dag(n, k, br)
    return sc, pi, edge


@pytest.mark.slow
def test_stationary_law_and_edge_posteriors():
    """The swap proposal is symmetric, so with the test ln u < ln10 * delta the chain's
    stationary law over orders is proportional to 10^score (Sec. III.C).  Check the
    lumped score distribution and the edge frequencies against exact enumeration of
    all 4! orders; the printed test without ln10 targets 10^(score/ln10) instead and
    must be told apart."""
    T, k = _small_problem()
    n = T.shape[0]
    sc, pi, edge = _exact(T, k)
    chains, iters, burn = 8, 40000, 1000
    out = oracle.mcmc_run(T, k, chains, iters, seed=7, burn_in=burn, trace=True)
    ts = out["trace_score"][:, burn:].ravel()
    # lumped distribution over distinct score values
    vals = np.unique(sc)
    emp = np.array([np.mean(ts == v) for v in vals])
    ex = np.array([pi[sc == v].sum() for v in vals])
    tv = 0.5 * np.abs(emp - ex).sum()
    assert tv < 0.02, (tv, emp, ex)
    f = out["edge_counts"].sum(axis=0) / (chains * (iters - burn))
    assert np.abs(f - edge).max() < 0.02
    # the literal (untempered) variant converges to a different law
    _, pi_lit, _ = _exact(T, k, temper=1.0 / math.log(10.0))
    lit = oracle.mcmc_run(T, k, chains, iters, seed=7, burn_in=burn, trace=True, literal_log=True)
    tl = lit["trace_score"][:, burn:].ravel()
    emp_l = np.array([np.mean(tl == v) for v in vals])
    ex_l = np.array([pi_lit[sc == v].sum() for v in vals])
    assert 0.5 * np.abs(emp_l - ex_l).sum() < 0.02
    assert 0.5 * np.abs(ex_l - ex).sum() > 0.05      # the two targets really differ


def test_trajectory_bookkeeping():
    T, k, *_ = (lambda d: (oracle.build_table(d[0], d[1], d[2], R=d[3]), d[2]))(
        synth.workload("n6_k2_m100"))
    n = T.shape[0]
    chains, iters, burn = 3, 500, 100
    out = oracle.mcmc_run(T, k, chains, iters, seed=11, burn_in=burn, trace=True)
    for c in range(chains):
        o0 = oracle.init_order(11, c, n)
        s0, _ = oracle.order_score(T, k, o0)
        acc = out["trace_accept"][c].astype(bool)
        assert out["accepts"][c] == acc.sum()
        # the best is the max over the initial state and the accepted states
        cand = np.concatenate([[s0], out["trace_score"][c][acc]])
        assert out["best_score"][c] == cand.max()
        sb, brb = oracle.order_score(T, k, out["best_order"][c])
        assert sb == out["best_score"][c] and (brb == out["best_rank"][c]).all()
        sf, _ = oracle.order_score(T, k, out["final_orders"][c])
        assert sf == out["final_score"][c] == out["trace_score"][c][-1]
        # rejected steps keep the score
        for t in range(1, iters):
            if not acc[t]:
                assert out["trace_score"][c][t] == out["trace_score"][c][t - 1]
        E = out["edge_counts"][c]
        assert E.max() <= iters - burn
        assert np.all(np.diag(E) == 0)


def test_ess_known_autocorrelation():
    rng = np.random.default_rng(0)
    T = 40000
    iid = rng.standard_normal(T)
    assert oracle.ess(iid) == pytest.approx(T, rel=0.1)
    for phi in (0.5, 0.9):
        x = np.zeros(T)
        e = rng.standard_normal(T)
        for t in range(1, T):
            x[t] = phi * x[t - 1] + e[t]
        # AR(1): integrated autocorrelation time (1 + phi) / (1 - phi)
        assert oracle.ess(x) == pytest.approx(T * (1 - phi) / (1 + phi), rel=0.15)
    assert math.isnan(oracle.ess(np.ones(100)))
    # a two-state Markov chain with flip probability p has lag-k correlation (1-2p)^k
    p = 0.1
    s = np.zeros(T)
    u = rng.random(T)
    for t in range(1, T):
        s[t] = 1 - s[t - 1] if u[t] < p else s[t - 1]
    lam = 1 - 2 * p
    assert oracle.ess(s) == pytest.approx(T * (1 - lam) / (1 + lam), rel=0.2)


def test_threaded_runs_equal_one_call():
    """The oracle's host-thread split (chains in contiguous groups, each group one call
    drawing the Philox streams of its own chain indices; the table's nodes in parallel)
    gives exactly what one single-threaded call gives."""
    data, arity, k, R, _ = synth.workload("n6_k2_m100")
    tab = oracle.build_table(data, arity, k, R=R)
    assert np.array_equal(tab, oracle.build_table(data, arity, k, R=R, threads=3))
    one = oracle.mcmc_run(tab, k, 7, 150, seed=11, burn_in=30, trace=True)
    for nt in (2, 3, 7):
        par = oracle.mcmc_run(tab, k, 7, 150, seed=11, burn_in=30, trace=True, threads=nt)
        for key in one:
            assert np.array_equal(one[key], par[key]), (nt, key)
    # chain0 selects the streams: chains 3..6 alone equal rows 3..6 of the full run
    tail = oracle.mcmc_run(tab, k, 4, 150, seed=11, burn_in=30, trace=True, chain0=3)
    for key in one:
        assert np.array_equal(one[key][3:], tail[key]), key
    orders = synth.random_orders(6, 9, 2)
    sc, br = oracle.order_scores(tab, k, orders, threads=4)
    for b in range(9):
        s, r = oracle.order_score(tab, k, orders[b])
        assert sc[b] == s and np.array_equal(br[b], r)
