"""The sum-based order score (the prior scorer of Sec. III.B) on the GPU against the
oracle's, which is pinned by enumerating every graph consistent with an order.  The two
sides add the same FP64 terms in different orders and evaluate 10^x with different
library routines, so the bar is 1e-12 relative per node term and per order."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,B", [("n6_k2_m100", 1), ("n6_k2_m100", 13), ("n20_k4_m1000", 9),
                                    ("n20_k4_m1000", 20)])
def test_sum_score_matches_oracle(gpu, name, B):
    data, arity, k, R, _ = synth.workload(name)
    n = data.shape[1]
    t = gpu.build_scores(data, arity, k, R=R)
    tab = gpu.table_scores(t)
    orders = synth.random_orders(n, B, 3 + B)
    sc, ns = gpu.score_orders_sum(t, orders)
    _, mx = gpu.score_orders(t, orders)
    for b in range(B):
        ref, ref_nodes = oracle.order_score_sum(tab, k, orders[b])
        np.testing.assert_allclose(ns[b], ref_nodes, rtol=1e-12, atol=1e-12)
        assert sc[b] == pytest.approx(ref, rel=1e-12)
        assert mx[b] <= sc[b] + 1e-9                      # log10 sum >= log10 max


def test_sum_score_full_size_sampled_n60(gpu):
    import torch
    data, arity, k, R, _ = synth.workload("n60_k4_m1000")
    t = gpu.build_scores(data, arity, k, R=R)
    tab = gpu.table_scores(t)
    orders = synth.random_orders(60, 3, 8)
    sc, ns = gpu.score_orders_sum(t, torch.as_tensor(orders, device="cuda"))
    sc, ns = sc.cpu().numpy(), ns.cpu().numpy()
    ref, ref_nodes = oracle.order_score_sum(tab, k, orders[0])
    np.testing.assert_allclose(ns[0], ref_nodes, rtol=1e-12, atol=1e-12)
    assert sc[0] == pytest.approx(ref, rel=1e-12)
    # the first node of every order has only the empty set
    for b in range(3):
        assert ns[b][orders[b][0]] == tab[orders[b][0], 0]
