"""The pruned scan (BN_SCAN_PRUNED) must give exactly the full scan's results: the same
ranks bit for bit and the same scores, in bn_score_orders and in the sampler; and the set
of surviving entries must be the one an independent dominance computation finds."""
import itertools

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _survivors_python(T, n, k):
    """Entries whose score beats every proper subset's (a separate restatement)."""
    S = T.shape[1]
    sets = [tuple(oracle.unrank(n - 1, k, r)) for r in range(S)]
    index = {s: r for r, s in enumerate(sets)}
    counts = []
    for i in range(n):
        best_le = np.empty(S)
        alive = 0
        for r, st in enumerate(sets):
            sub = max((best_le[index[st[:t] + st[t + 1:]]] for t in range(len(st))), default=-np.inf)
            best_le[r] = max(T[i, r], sub)
            alive += T[i, r] > sub
        counts.append(alive)
    return np.array(counts)


@pytest.mark.parametrize("name", ["n6_k2_m100", "n20_k4_m1000"])
def test_survivors_match_python_dominance(gpu, name):
    data, arity, k, R, _ = synth.workload(name)
    n = data.shape[1]
    t = gpu.build_scores(data, arity, k, R=R)
    T = gpu.table_scores(t)
    gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    assert np.array_equal(gpu.table_pruned(t), _survivors_python(T, n, k))


@pytest.mark.parametrize("name,B", [("n6_k2_m100", 100), ("n20_k4_m1000", 300), ("n40_k4_m2000", 512),
                                    ("n60_k4_m1000", 256)])
def test_pruned_equals_full(gpu, name, B):
    data, arity, k, R, _ = synth.workload(name)
    n = data.shape[1]
    t = gpu.build_scores(data, arity, k, R=R)
    orders = synth.random_orders(n, B, 21)
    br_f, sc_f = gpu.score_orders(t, orders)
    gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    br_p, sc_p = gpu.score_orders(t, orders)
    assert np.array_equal(br_f, br_p)
    assert np.array_equal(sc_f, sc_p)
    surv = gpu.table_pruned(t)
    assert (surv >= 1).all() and surv.sum() < t.info()["sets_per_node"] * n


def test_pruned_all_720_orders_vs_oracle(gpu):
    data, arity, k, R, _ = synth.workload("n6_k2_m100", 1)
    tab = oracle.build_table(data, arity, k)
    t = gpu.table_from_scores(tab, k)
    gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    orders = np.array(list(itertools.permutations(range(6))), np.uint8)
    br, sc = gpu.score_orders(t, orders)
    for b, o in enumerate(orders):
        s, r = oracle.order_score(tab, k, o)
        assert np.array_equal(br[b], r) and sc[b] == s


def test_pruned_ties(gpu):
    # every entry equal: everything but the empty set is dominated
    n, k = 8, 3
    tab = np.zeros((n, oracle.num_sets(n - 1, k)))
    t = gpu.table_from_scores(tab, k)
    gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    assert (gpu.table_pruned(t) == 1).all()
    br, sc = gpu.score_orders(t, synth.random_orders(n, 50, 2))
    assert (br == 0).all() and (sc == 0).all()


def test_pruned_sampler_trajectories_vs_oracle(gpu):
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    tab = oracle.build_table(data, arity, k, R=R)
    t = gpu.table_from_scores(tab, k)
    gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    ch = gpu.chains_create(t, 8, 31, burn_in=50, trace_cap=300)
    gpu.chains_step(ch, 300)
    ref = oracle.mcmc_run(tab, k, 8, 300, seed=31, burn_in=50, trace=True)
    assert np.array_equal(gpu.chains_read(ch, "trace_score"), ref["trace_score"])
    assert np.array_equal(gpu.chains_read(ch, "edge_counts").astype(np.uint64), ref["edge_counts"])


def test_fused_steps_equal_batched_steps(gpu):
    """Uniform proposals on a pruned table run as fused multi-step launches (one warp
    per chain); every output must equal the per-step batched path on the full table."""
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    t = gpu.build_scores(data, arity, k, R=R)
    kw = dict(burn_in=30, record_every=3, record_cap=200, trace_cap=600)
    a = gpu.chains_create(t, 64, 4242, **kw)
    gpu.chains_step(a, 600)                                  # batched, full scan
    gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    b = gpu.chains_create(t, 64, 4242, **kw)
    for s in (100, 7, 300, 193):                             # fused, across chunk boundaries
        gpu.chains_step(b, s)
    for what in ("trace_score", "trace_accept", "orders", "scores", "ranks", "best_orders", "best_scores",
                 "best_ranks", "accepts", "edge_counts", "record", "record_len", "steps", "items"):
        assert np.array_equal(gpu.chains_read(a, what), gpu.chains_read(b, what)), what
    ea, eb = gpu.chains_read(a, "ess"), gpu.chains_read(b, "ess")
    assert np.array_equal(np.isnan(ea), np.isnan(eb)) and np.allclose(ea[~np.isnan(ea)], eb[~np.isnan(eb)])


@pytest.mark.parametrize("trace_cap", [0, 150])
def test_fused_untraced_equals_batched_steps(gpu, trace_cap):
    """Without per-step score traces the fused kernel leaves the FP64 score of moves its
    fast test accepts for later, tracks the state by the exact fixed-point sum and decides
    new bests in fixed point where that is provably the same decision; every output must
    still equal the per-step path (which sums every accepted score in FP64), bit for bit.
    Long enough that chains return to their best states and leave them again."""
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    t = gpu.build_scores(data, arity, k, R=R)
    kw = dict(burn_in=100, record_every=7, record_cap=400, trace_cap=trace_cap)
    a = gpu.chains_create(t, 64, 5151, **kw)
    gpu.chains_step(a, 1500)                                 # batched, full scan
    gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    b = gpu.chains_create(t, 64, 5151, **kw)
    for s in (500, 77, 923):                                 # fused, across chunk boundaries
        gpu.chains_step(b, s)
    outs = ["orders", "scores", "ranks", "best_orders", "best_scores", "best_ranks", "accepts", "edge_counts",
            "record", "record_len", "steps", "items"]
    if trace_cap:
        outs += ["trace_score", "trace_accept"]
    for what in outs:
        assert np.array_equal(gpu.chains_read(a, what), gpu.chains_read(b, what)), what


def test_switching_mode_recaptures_the_step(gpu):
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    t = gpu.build_scores(data, arity, k, R=R)
    a = gpu.chains_create(t, 16, 8, trace_cap=200)
    gpu.chains_step(a, 100)
    gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    gpu.chains_step(a, 100)
    gpu.table_set_scan(t, gpu.SCAN_FULL)
    b = gpu.chains_create(t, 16, 8, trace_cap=200)
    gpu.chains_step(b, 200)
    assert np.array_equal(gpu.chains_read(a, "trace_score"), gpu.chains_read(b, "trace_score"))


@pytest.mark.parametrize("trace_cap", [400, 0])
def test_fused_steps_equal_batched_steps_uncached_survivors(gpu, trace_cap):
    """A network with more survivors than the shared-memory cache holds (little data: many
    parent sets stay undominated) runs on the same cache layout in global memory; results
    must still equal the per-step path on the full table, bit for bit."""
    ar = np.full(50, 3, np.uint8)
    net = synth.random_network(50, 3, ar, 0xB4E5_0B0B)
    data = synth.forward_sample(net, 250, 0xB4E5_0B0C)
    t = gpu.build_scores(data, ar, 4)
    kw = dict(burn_in=20, trace_cap=trace_cap)
    a = gpu.chains_create(t, 32, 99, **kw)
    gpu.chains_step(a, 400)
    gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    assert gpu.table_pruned(t).sum() > 2400
    b = gpu.chains_create(t, 32, 99, **kw)
    gpu.chains_step(b, 150)
    gpu.chains_step(b, 250)
    outs = ["orders", "ranks", "scores", "best_scores", "best_orders", "best_ranks", "accepts", "edge_counts"]
    if trace_cap:
        outs += ["trace_score", "trace_accept"]
    for what in outs:
        assert np.array_equal(gpu.chains_read(a, what), gpu.chains_read(b, what)), what


@pytest.mark.parametrize("trace_cap", [0, 400])
def test_fused_fallback_for_large_entries_equals_batched(gpu, trace_cap):
    """Entries beyond the fused kernel's fixed-point range (|entry| >= 2^22; here every
    entry shifted by -1e7, which changes no order and no dominance) take its fallback,
    which re-scores every span node from the table's survivor arrays with FP64 changes."""
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    sc = gpu.table_scores(gpu.build_scores(data, arity, k, R=R)) - 1.0e7
    t = gpu.table_from_scores(sc, k)
    kw = dict(burn_in=30, trace_cap=trace_cap, record_every=5, record_cap=100)
    a = gpu.chains_create(t, 32, 11, **kw)
    gpu.chains_step(a, 400)                                  # batched, full scan
    gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    b = gpu.chains_create(t, 32, 11, **kw)
    gpu.chains_step(b, 150)
    gpu.chains_step(b, 250)
    outs = ["orders", "scores", "ranks", "best_orders", "best_scores", "best_ranks", "accepts", "edge_counts",
            "record", "steps", "items"]
    if trace_cap:
        outs += ["trace_score", "trace_accept"]
    for what in outs:
        assert np.array_equal(gpu.chains_read(a, what), gpu.chains_read(b, what)), what
