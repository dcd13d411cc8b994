"""The accuracy study of Sec. VI on the library: the best graph of the 20-node workload
against its true DAG (ROC points), the effect of a prior built from the prior-free run's
errors, and the effect of flipping noise in binary data.  The first tests check
properties of the method on seeded data, so their bars are loose: the learned graph
recovers most true edges with few false ones, a decisive prior on the prior-free run's
errors corrects them, and heavy noise costs true positives.  The last two run the same
study's single-chain learning runs on the oracle (its own table and sampler, same seeds)
and require the identical best graph."""
import numpy as np
import pytest

import oracle
import synth
from paper_1210_5128_gb300 import roc

pytestmark = pytest.mark.gpu


def _learn(gpu, data, arity, k, R, iters, seed, chains=1):
    t = gpu.build_scores(data, arity, k, R=R)
    gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    return gpu.mcmc_run(t, chains, iters, seed=seed, burn_in=iters // 10)["best_dag"]


def test_roc_points_and_prior_n20(gpu):
    data, arity, k, _, net = synth.workload("n20_k4_m1000")
    T = roc.true_adjacency(net)
    L = _learn(gpu, data, arity, k, None, 10000, 3, chains=16)
    tp, fp = roc.tp_fp(L, T)
    assert tp >= 0.5 and fp <= 0.05, (tp, fp)
    tp_s, fp_s = roc.tp_fp(L, T, skeleton=True)
    assert tp_s >= tp
    # a decisive prior on every error of the prior-free run (R = 1 on missed edges, 0 on
    # wrongly added ones: +-12.5 per parent set) must correct them, and cost nothing else
    Rp = roc.prior_from_errors(L, T, 1.0, 0.0, 1.0, seed=1)
    L2 = _learn(gpu, data, arity, k, Rp, 10000, 3, chains=16)
    target = Rp != 0.5
    if target.any():
        fixed = (L2.astype(bool) == T.astype(bool))[target].mean()
        assert fixed >= 0.9, fixed
    tp2, fp2 = roc.tp_fp(L2, T)
    assert tp2 >= tp - 0.05 and fp2 <= fp + 0.01, ((tp, fp), (tp2, fp2))


def test_noise_costs_true_positives_binary_n20(gpu):
    net = synth.random_network(20, 3, 2, 0xB4E5_0A0A)
    data = synth.forward_sample(net, 1000, 0xB4E5_0A0B)
    T = roc.true_adjacency(net)
    ar = np.full(20, 2, np.uint8)
    tp0, _ = roc.tp_fp(_learn(gpu, data, ar, 4, None, 10000, 5, chains=16), T)
    tp1, _ = roc.tp_fp(_learn(gpu, roc.flip_noise(data, 0.15, 7), ar, 4, None, 10000, 5, chains=16), T)
    assert tp1 <= tp0, (tp0, tp1)


def _learn_both(gpu, data, arity, k, R, iters, seed):
    """One chain on the library (its own table, pruned, fused sampler) and on the oracle
    (its own table, brute-force order scores): best DAG and best score of each."""
    n = data.shape[1]
    t = gpu.build_scores(data, arity, k, R=R)
    gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    out = gpu.mcmc_run(t, 1, iters, seed=seed, burn_in=iters // 10)
    tab = oracle.build_table(data, arity, k, R=R, threads=None)
    ref = oracle.mcmc_run(tab, k, 1, iters, seed=seed, burn_in=iters // 10)
    return out, oracle.greedy_dag(n, k, ref["best_rank"][0]), float(ref["best_score"][0])


def _same_point(gpu_out, ref_dag, ref_score, T):
    assert np.array_equal(gpu_out["best_dag"], ref_dag)
    assert abs(gpu_out["best_score"] - ref_score) <= 1e-9 * abs(ref_score)
    assert roc.tp_fp(gpu_out["best_dag"], T) == roc.tp_fp(ref_dag, T)


def test_roc_points_against_oracle(gpu):
    """The ROC study's runs (one chain, 1,000 and 10,000 iterations; a prior schedule point
    built from the prior-free run's errors) give the oracle's best graph exactly."""
    data, arity, k, _, net = synth.workload("n20_k4_m1000")
    T = roc.true_adjacency(net)
    ref_free = {}
    for iters in (1000, 10000):
        out, ref_dag, ref_score = _learn_both(gpu, data, arity, k, None, iters, 29)
        _same_point(out, ref_dag, ref_score, T)
        ref_free[iters] = ref_dag
    Rp = roc.prior_from_errors(ref_free[1000], T, 0.7, 0.2, 0.4, seed=31)
    assert (Rp != 0.5).any()
    out, ref_dag, ref_score = _learn_both(gpu, data, arity, k, Rp, 1000, 29)
    _same_point(out, ref_dag, ref_score, T)


def test_noise_point_against_oracle(gpu):
    """A noise-study point (binary data, every value flipped with probability 0.1)."""
    net = synth.random_network(20, 3, 2, 0xB4E5_0A0A)
    data = roc.flip_noise(synth.forward_sample(net, 1000, 0xB4E5_0A0B), 0.1, 46)
    out, ref_dag, ref_score = _learn_both(gpu, data, np.full(20, 2, np.uint8), 4, None, 3000, 29)
    _same_point(out, ref_dag, ref_score, roc.true_adjacency(net))
