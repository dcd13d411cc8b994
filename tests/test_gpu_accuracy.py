"""The accuracy study of Sec. VI on the library: the best graph of the 20-node workload
against its true DAG (ROC points), the effect of a prior built from the prior-free run's
errors, and the effect of flipping noise in binary data.  These are properties of the
method on seeded data, so the bars are loose: the learned graph recovers most true edges
with few false ones, a decisive prior on the prior-free run's errors corrects them, and
heavy noise costs true positives."""
import numpy as np
import pytest

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
