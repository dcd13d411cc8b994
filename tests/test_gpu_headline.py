"""The headline sampler at its own sizes against the oracle (Algorithm 1, Eq. 6).

The fused kernel that advances every chain up to 1,024 MH steps per launch with the
network's surviving parent sets staged in shared memory is checked here at n = 40 and
n = 60 (k = 4), where a swap's span can exceed the 32 lanes of a warp (lane l then holds
span positions a + l and a + l + 32):

- n = 40: traced and untraced runs against the oracle's own sampler on the oracle's own
  table, step for step (scores, accept flags, final and best states, edge counts), with
  the survivors in shared memory (m = 1000) and in the cache's global-memory copy
  (m = 2000, more survivors than shared memory holds);
- n = 60: the bench's shape, 256 chains in two untraced 1,000-step launches, against the
  full-table sampler (three kernels per step, no pruning) bit for bit, the final and
  best orders of a sample of chains re-scored by the oracle, and the first steps of 16
  chains against the oracle's trajectories.

The tables are the workloads' own (n = 40: 3 states, m = 1000 and 2000; n = 60: 3 states,
m = 1000, the bench's table), every entry built by the oracle on the host's cores; the
n = 60 one is also compared with the GPU's build of the same data, every entry."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SURV_CACHE_MAX = 2400          # survivors a network may have for the shared-memory cache
OUTS = ("orders", "scores", "ranks", "best_scores", "best_orders", "best_ranks", "accepts", "edge_counts",
        "steps", "items")


def _spans(n, seed, chains, steps):
    """Span lengths b - a + 1 of the uniform swaps the Philox streams draw (the fixed
    definition both sides follow), chains x steps."""
    P = n * (n - 1) // 2
    out = np.zeros((chains, steps), np.int64)
    for c in range(chains):
        for t in range(steps):
            x = oracle.philox4x64([t, c, 0, 0], [seed, 0])
            a, b = oracle.pair_decode(n, (int(x[0]) * P) >> 64)
            out[c, t] = b - a + 1
    return out


def _pruned(gpu, tab, k, staged=True):
    """The oracle's table, pruned; staged: its survivors fit the fused kernel's
    shared-memory cache (else they run from the global-memory copy of the cache)."""
    t = gpu.table_from_scores(tab, k)
    gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    surv = int(gpu.table_pruned(t).sum())
    assert surv > 0 and (surv <= SURV_CACHE_MAX) == staged, surv
    return t


@pytest.mark.parametrize("which,staged", [("oracle_n40_m1000", True), ("oracle_n40", False)])
def test_n40_fused_sampler_against_oracle(gpu, request, which, staged):
    """n = 40 with 1,000 samples (survivors in shared memory) and with 2,000 samples (more
    survivors than the shared-memory cache holds: the same walk over the cache's
    global-memory copy)."""
    data, arity, k, R, tab = request.getfixturevalue(which)
    n = tab.shape[0]
    chains, steps, seed, burn = 8, 60, 4040, 10
    assert (_spans(n, seed, chains, steps) > 32).sum() >= 5      # the lane-half path runs
    t = _pruned(gpu, tab, k, staged)
    ref = oracle.mcmc_run(tab, k, chains, steps, seed=seed, burn_in=burn, trace=True, threads=None)
    traced = gpu.chains_create(t, chains, seed, burn_in=burn, trace_cap=steps)
    gpu.chains_step(traced, steps)
    untraced = gpu.chains_create(t, chains, seed, burn_in=burn)
    gpu.chains_step(untraced, steps)
    assert np.array_equal(gpu.chains_read(traced, "trace_score"), ref["trace_score"])
    assert np.array_equal(gpu.chains_read(traced, "trace_accept"), ref["trace_accept"])
    for ch in (traced, untraced):
        assert np.array_equal(gpu.chains_read(ch, "orders"), ref["final_orders"])
        assert np.array_equal(gpu.chains_read(ch, "scores"), ref["final_score"])
        assert np.array_equal(gpu.chains_read(ch, "best_scores"), ref["best_score"])
        assert np.array_equal(gpu.chains_read(ch, "best_orders"), ref["best_order"])
        assert np.array_equal(gpu.chains_read(ch, "best_ranks"), ref["best_rank"])
        assert np.array_equal(gpu.chains_read(ch, "accepts"), ref["accepts"])
        assert np.array_equal(gpu.chains_read(ch, "edge_counts").astype(np.uint64), ref["edge_counts"])
    assert ref["accepts"].sum() > 0


def test_n60_table_every_entry(gpu, oracle_n60):
    data, arity, k, R, tab = oracle_n60
    t = gpu.build_scores(data, arity, k, R=R)
    np.testing.assert_allclose(gpu.table_scores(t), tab, rtol=1e-12, atol=1e-12)


def test_n60_first_steps_against_oracle(gpu, oracle_n60):
    """16 chains, 5 steps each, traced, against the oracle's trajectories (an oracle step
    at n = 60 is a full brute-force order score, about a second of CPU time)."""
    _, _, k, _, tab = oracle_n60
    n = tab.shape[0]
    chains, steps, seed = 16, 5, 6060
    assert (_spans(n, seed, chains, steps) > 32).sum() >= 5
    t = _pruned(gpu, tab, k)
    ch = gpu.chains_create(t, chains, seed, trace_cap=steps)
    gpu.chains_step(ch, steps)
    ref = oracle.mcmc_run(tab, k, chains, steps, seed=seed, trace=True, threads=None)
    assert np.array_equal(gpu.chains_read(ch, "trace_score"), ref["trace_score"])
    assert np.array_equal(gpu.chains_read(ch, "trace_accept"), ref["trace_accept"])
    assert np.array_equal(gpu.chains_read(ch, "orders"), ref["final_orders"])
    assert np.array_equal(gpu.chains_read(ch, "best_ranks"), ref["best_rank"])


def test_n60_headline_launches_equal_full_table_and_oracle(gpu, oracle_n60):
    """The bench's shape: 256 chains, untraced, two 1,000-step calls (one fused launch
    each) against the unpruned full-table sampler over the same 2,000 steps."""
    _, _, k, _, tab = oracle_n60
    n = tab.shape[0]
    chains, seed, burn = 256, 60256, 100
    spans = _spans(n, seed, 2, 200)
    assert (spans > 32).mean() > 0.1
    full_t = gpu.table_from_scores(tab, k)
    full = gpu.chains_create(full_t, chains, seed, burn_in=burn)
    gpu.chains_step(full, 2000)
    t = _pruned(gpu, tab, k)
    fused = gpu.chains_create(t, chains, seed, burn_in=burn)
    for _ in range(2):
        gpu.chains_step(fused, 1000)
    for what in OUTS:
        assert np.array_equal(gpu.chains_read(fused, what), gpu.chains_read(full, what)), what
    assert gpu.chains_read(fused, "accepts").min() > 0
    # the oracle re-scores the final and best orders of a sample of chains: the GPU's
    # ranks and FP64 scores of those states must be its ranks and sums exactly
    pick = np.random.default_rng(3).choice(chains, 8, replace=False)
    orders = np.concatenate([gpu.chains_read(fused, "orders")[pick], gpu.chains_read(fused, "best_orders")[pick]])
    sc, br = oracle.order_scores(tab, k, orders)
    assert np.array_equal(br[:8], gpu.chains_read(fused, "ranks")[pick])
    assert np.array_equal(sc[:8], gpu.chains_read(fused, "scores")[pick])
    assert np.array_equal(br[8:], gpu.chains_read(fused, "best_ranks")[pick])
    assert np.array_equal(sc[8:], gpu.chains_read(fused, "best_scores")[pick])
    # edge counts: every post-burn-in step counts each edge of the current greedy DAG once
    E = gpu.chains_read(fused, "edge_counts")
    assert (E.sum((1, 2)) <= 2000 * n * k).all() and (np.diagonal(E, axis1=1, axis2=2) == 0).all()


@pytest.mark.parametrize("B", [4, 8, 16, 17, 136, 137, 1024])
def test_n60_batched_scoring_against_oracle(gpu, oracle_n60, B):
    """bn_score_orders at the bench's table on the oracle's entries: the scan of all
    nodes' rank range with up to eight orders a thread (n * ceil(B / 8) <= 1,024 items:
    B = 4, 8, 16 with several threads an item, B = 17 and 136 one thread an item, 136 in
    1,024-thread blocks), the full-table scan (B = 137, 1,024; autotuned tiling) and the
    pruned table give the same ranks and FP64 sums, and a sample of orders equals the
    oracle's brute-force order score."""
    _, _, k, _, tab = oracle_n60
    orders = synth.random_orders(60, B, 1700 + B)
    full = gpu.table_from_scores(tab, k)
    br_f, sc_f = gpu.score_orders(full, orders)
    pruned = gpu.table_from_scores(tab, k)
    gpu.table_set_scan(pruned, gpu.SCAN_PRUNED)
    br_p, sc_p = gpu.score_orders(pruned, orders)
    assert np.array_equal(br_f, br_p) and np.array_equal(sc_f, sc_p)
    pick = sorted(set([0, B - 1] + list(np.random.default_rng(B).choice(B, min(B, 14), replace=False))))
    sc_ref, br_ref = oracle.order_scores(tab, k, orders[pick])
    assert np.array_equal(br_f[pick], br_ref)
    assert np.array_equal(sc_f[pick], sc_ref)
