"""The learned proposal's step path on a pruned table: one warp per chain for the MH
bookkeeping and the network's first layer (fixed-point sums of per-(position, node) rows),
two tcgen05 kernels for the dense layers, three launches per step in a CUDA graph.

- network outputs: the logits held for every chain's current order match the FP64 oracle
  of the network on the same bf16 rounding points (the bar of the network's own forward
  test), before and after steps, at a ragged number of chains;
- path independence: after steps, the logits equal bit for bit those computed from
  scratch for the same orders by a fresh chain set (q(. | order) is a function of the order);
- chain state: every chain's score is the oracle's order score of its order (relative
  1e-9) with the oracle's argmax parent sets, bit for bit;
- the posterior and the useful-move gain are tested on both paths in test_gpu_learned."""
import numpy as np
import pytest

import oracle
import synth
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def _weights(n, d, H, seed, sharpen=1.0):
    w = synth.mlp_init_weights(n, d, H, seed)
    w["W3"] = (w["W3"] * sharpen).astype(np.float32)
    return w, omlp.MLPParams(*(np.asarray(w[k], np.float64) for k in ["E", "W1", "b1", "W2", "b2", "W3", "b3"]))


def _close(a, b, elem=1e-2, norm=1e-3):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = max(np.abs(b).max(), 1e-30)
    assert np.abs(a - b).max() <= elem * scale, (np.abs(a - b).max(), scale)
    assert np.linalg.norm(a - b) <= norm * max(np.linalg.norm(b), 1e-30) + 1e-30


@pytest.mark.parametrize("name,d,H,C", [("n20_k4_m1000", 32, 256, 200), ("n60_k4_m1000", 32, 512, 256)])
def test_logits_match_oracle_and_depend_on_the_order_alone(gpu, name, d, H, C):
    data, arity, k, R, _ = synth.workload(name)
    n = data.shape[1]
    t = gpu.build_scores(data, arity, k, R=R)
    gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    w, prm = _weights(n, d, H, 11, sharpen=4.0)
    net = gpu.mlp_create(n, w, hidden=H, d=d, batch_cap=C)
    ch = gpu.chains_create(t, C, 31)
    gpu.chains_step(ch, 40)
    gpu.chains_set_proposal(ch, net, gpu.PROPOSAL_LEARNED, eps_mix=0.1)
    O = gpu.chains_read(ch, "orders")
    _close(gpu.chains_read(ch, "logits"), omlp.mlp_forward(prm, O)["logits"])
    a0 = gpu.chains_read(ch, "accepts").copy()
    gpu.chains_step(ch, 150)
    assert (gpu.chains_read(ch, "accepts") > a0).mean() > 0.5      # most chains moved
    O2 = gpu.chains_read(ch, "orders")
    L2 = gpu.chains_read(ch, "logits")
    _close(L2, omlp.mlp_forward(prm, O2)["logits"])
    # the same orders primed from scratch give the same bits
    fresh = gpu.chains_create(t, C, 77, init_orders=O2)
    gpu.chains_set_proposal(fresh, net, gpu.PROPOSAL_LEARNED, eps_mix=0.1)
    assert np.array_equal(gpu.chains_read(fresh, "logits"), L2)


@pytest.mark.parametrize("name,C,steps", [("n6_k2_m100", 37, 300), ("n20_k4_m1000", 130, 200)])
def test_chain_state_matches_oracle(gpu, name, C, steps):
    data, arity, k, R, _ = synth.workload(name)
    n = data.shape[1]
    t = gpu.build_scores(data, arity, k, R=R)
    tab = gpu.table_scores(t)
    gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    d, H = 8, 128
    w, _ = _weights(n, d, H, 3, sharpen=6.0)
    net = gpu.mlp_create(n, w, hidden=H, d=d, batch_cap=C)
    ch = gpu.chains_create(t, C, 5, trace_cap=steps)
    gpu.chains_set_proposal(ch, net, gpu.PROPOSAL_LEARNED, eps_mix=0.2)
    gpu.chains_step(ch, steps // 2)
    gpu.chains_step(ch, steps - steps // 2)                 # two calls: state carried across
    assert gpu.chains_read(ch, "steps")[0] == steps
    O = gpu.chains_read(ch, "orders")
    sc = gpu.chains_read(ch, "scores")
    rk = gpu.chains_read(ch, "ranks")
    acc = gpu.chains_read(ch, "accepts")
    tr = gpu.chains_read(ch, "trace_score")
    ta = gpu.chains_read(ch, "trace_accept")
    assert np.array_equal(acc, ta.sum(1).astype(np.int64))
    assert np.array_equal(tr[:, -1], sc)
    for c in range(0, C, max(1, C // 12)):
        assert sorted(O[c]) == list(range(n))
        s_ref, br_ref = oracle.order_score(tab, k, O[c])
        assert sc[c] == pytest.approx(s_ref, rel=1e-9, abs=1e-9)
        assert np.array_equal(rk[c], br_ref)
    # the best score seen is at least every traced score of the chain
    best = gpu.chains_read(ch, "best_scores")
    assert (best[:, None] >= tr - 1e-9 * np.abs(tr)).all()
    bo, bs = gpu.chains_read(ch, "best_orders"), best
    for c in range(0, C, max(1, C // 6)):
        assert oracle.order_score(tab, k, bo[c])[0] == pytest.approx(bs[c], rel=1e-9, abs=1e-9)


def test_uniform_steps_between_learned_calls(gpu):
    """Uniform steps move the orders outside the learned path; the next learned call must
    re-derive its layer-1 sums and outputs for the moved orders."""
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    n = data.shape[1]
    t = gpu.build_scores(data, arity, k, R=R)
    gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    w, prm = _weights(n, 16, 128, 8, sharpen=3.0)
    net = gpu.mlp_create(n, w, hidden=128, d=16, batch_cap=64)
    ch = gpu.chains_create(t, 64, 9)
    gpu.chains_set_proposal(ch, net, gpu.PROPOSAL_LEARNED, eps_mix=0.1)
    gpu.chains_step(ch, 30)
    gpu.chains_set_proposal(ch, None, gpu.PROPOSAL_UNIFORM)
    gpu.chains_step(ch, 300)
    gpu.chains_set_proposal(ch, net, gpu.PROPOSAL_LEARNED, eps_mix=0.1)
    gpu.chains_step(ch, 30)
    O = gpu.chains_read(ch, "orders")
    _close(gpu.chains_read(ch, "logits"), omlp.mlp_forward(prm, O)["logits"])
    tab = gpu.table_scores(t)
    sc = gpu.chains_read(ch, "scores")
    for c in range(0, 64, 9):
        assert sc[c] == pytest.approx(oracle.order_score(tab, k, O[c])[0], rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("name,d,H,C,steps", [("n6_k2_m100", 8, 128, 37, 300), ("n20_k4_m1000", 32, 256, 200, 600),
                                              ("n60_k4_m1000", 32, 512, 256, 300)])
def test_persistent_launch_equals_graph_launch(gpu, name, d, H, C, steps):
    """The persistent cooperative kernel (the three phases of each step separated by
    grid-wide barriers, up to 256 steps per launch) gives bit for bit what the three
    kernels per step replayed from a CUDA graph give: traces, states, best states, edge
    counts, records and the network outputs held for the final orders."""
    data, arity, k, R, _ = synth.workload(name)
    n = data.shape[1]
    t = gpu.build_scores(data, arity, k, R=R)
    gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    w, _ = _weights(n, d, H, 21, sharpen=4.0)
    out = []
    for mode in (gpu.LEARNED_LAUNCH_GRAPH, gpu.LEARNED_LAUNCH_AUTO):
        net = gpu.mlp_create(n, w, hidden=H, d=d, batch_cap=C)
        ch = gpu.chains_create(t, C, 41, burn_in=50, trace_cap=steps, record_every=3, record_cap=steps)
        gpu.chains_set_learned_launch(ch, mode)
        gpu.chains_step(ch, 20)
        gpu.chains_set_proposal(ch, net, gpu.PROPOSAL_LEARNED, eps_mix=0.15)
        gpu.chains_step(ch, steps // 3)
        gpu.chains_step(ch, steps - 20 - steps // 3)
        out.append({what: gpu.chains_read(ch, what) for what in
                    ("trace_score", "trace_accept", "orders", "scores", "ranks", "best_scores", "best_orders",
                     "best_ranks", "accepts", "edge_counts", "steps", "items", "record", "record_len", "logits")})
    for what in out[0]:
        assert np.array_equal(out[0][what], out[1][what]), what
    assert out[1]["accepts"].sum() > 0
