"""The learned swap proposal inside the MH ratio.

Exactness: with any proposal network (here a random, far-from-uniform one) the chain
must still sample the order posterior proportional to 10^score, so its edge frequencies
must match the exact edge posteriors obtained by enumerating all 720 orders of the
6-node workload with the oracle.  Gain: after training on the uniform sampler's own
history the learned proposal must get its swaps accepted more often than uniform swaps."""
import itertools

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _exact_edge_posterior(tab, k):
    n = tab.shape[0]
    orders = [np.array(o, np.uint8) for o in itertools.permutations(range(n))]
    res = [oracle.order_score(tab, k, o) for o in orders]
    sc = np.array([r[0] for r in res])
    w = np.power(10.0, sc - sc.max())
    w /= w.sum()
    post = np.zeros((n, n))
    for (s, br), p in zip(res, w):
        post += p * oracle.greedy_dag(n, k, br)
    return post


@pytest.mark.parametrize("scan", ["full", "pruned"])
def test_learned_proposal_keeps_the_posterior_n6(gpu, scan):
    data, arity, k, R, _ = synth.workload("n6_k2_m100", 7)
    # a flatter posterior (fewer samples) so several orders carry weight
    data = data[:30].copy()
    tab = oracle.build_table(data, arity, k)
    exact = _exact_edge_posterior(tab, k)
    n, d, H = 6, 8, 128
    w = synth.mlp_init_weights(n, d, H, 3)
    w["W3"] *= 8.0                                  # strongly non-uniform pair preferences
    w["b3"] = np.linspace(-3, 3, n * (n - 1) // 2).astype(np.float32)
    net = gpu.mlp_create(n, w, hidden=H, d=d, batch_cap=128)
    t = gpu.table_from_scores(tab, k)
    if scan == "pruned":                  # the three-kernel learned step path
        gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    C, steps, burn = 128, 6000, 500
    ch = gpu.chains_create(t, C, 99, burn_in=burn)
    gpu.chains_set_proposal(ch, net, gpu.PROPOSAL_LEARNED, eps_mix=0.2)
    gpu.chains_step(ch, steps)
    f = gpu.chains_read(ch, "edge_counts").sum(0) / (C * (steps - burn))
    assert np.abs(f - exact).max() < 0.02, np.abs(f - exact).max()
    # the proposal really was far from uniform: its pair probabilities span more than a
    # factor of 5 on the chains' final orders
    logits = gpu.mlp_forward(net, gpu.chains_read(ch, "orders"))
    q = 0.8 * np.exp(logits - logits.max(1, keepdims=True))
    q = q / (q.sum(1, keepdims=True) / 0.8) + 0.2 / logits.shape[1]
    assert (q.max(1) / q.min(1)).min() > 5.0
    # the uniform sampler agrees with the same posterior
    u = gpu.chains_create(t, C, 99, burn_in=burn)
    gpu.chains_step(u, steps)
    fu = gpu.chains_read(u, "edge_counts").sum(0) / (C * (steps - burn))
    assert np.abs(fu - exact).max() < 0.02


@pytest.mark.parametrize("scan", ["full", "pruned"])
def test_training_on_history_raises_the_rate_of_useful_moves_n20(gpu, scan):
    """The network is trained to propose swaps that are accepted AND change the graph
    (swaps that change no parent set are always accepted but move nothing).  After
    training, the fraction of steps whose order score actually changes must be higher
    with the learned proposal than with uniform swaps from the same states."""
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    t = gpu.build_scores(data, arity, k, R=R)
    if scan == "pruned":
        gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    n, d, H = 20, 32, 256
    net = gpu.mlp_create(n, synth.mlp_init_weights(n, d, H, 4), hidden=H, d=d, batch_cap=256, lr=2e-3)
    C, burn, train, m = 256, 200, 600, 300
    ch = gpu.chains_create(t, C, 5, trace_cap=burn + train + 2 * m)
    gpu.chains_step(ch, burn)                                    # burn in with uniform swaps
    gpu.chains_set_proposal(ch, net, gpu.PROPOSAL_TRAIN)
    gpu.chains_step(ch, train)                                   # train on the chains' history
    gpu.chains_set_proposal(ch, None, gpu.PROPOSAL_UNIFORM)
    gpu.chains_step(ch, m)
    gpu.chains_set_proposal(ch, net, gpu.PROPOSAL_LEARNED, eps_mix=0.1)
    gpu.chains_step(ch, m)
    tr = gpu.chains_read(ch, "trace_score")
    moved = tr[:, 1:] != tr[:, :-1]
    s0 = burn + train
    useful_uniform = moved[:, s0:s0 + m - 1].mean()
    useful_learned = moved[:, s0 + m:s0 + 2 * m - 1].mean()
    assert useful_learned > 1.2 * useful_uniform, (useful_learned, useful_uniform)
