"""GPU parity of the MH swap sampler (Sec. III.C) against the oracle on a shared table:
the same Philox draws, so trajectories, acceptances, best graphs and edge counts must be
identical step for step (a decision could only differ if ln u and ln10 * delta agree to
within rounding, which these seeds do not hit)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _shared(name="n6_k2_m100", off=0):
    data, arity, k, R, _ = synth.workload(name, off)
    return oracle.build_table(data, arity, k, R=R), k


def _run_both(gpu, tab, k, chains, steps, seed, burn_in=0, literal=False):
    t = gpu.table_from_scores(tab, k)
    ch = gpu.chains_create(t, chains, seed, burn_in=burn_in, trace_cap=steps, literal_log=literal)
    init = gpu.chains_read(ch, "orders")
    gpu.chains_step(ch, steps)
    ref = oracle.mcmc_run(tab, k, chains, steps, seed=seed, burn_in=burn_in, trace=True,
                          literal_log=literal)
    return ch, init, ref


@pytest.mark.parametrize("name,chains,steps", [("n6_k2_m100", 3, 400), ("n20_k4_m1000", 8, 300)])
def test_trajectories_identical(gpu, name, chains, steps):
    tab, k = _shared(name)
    ch, init, ref = _run_both(gpu, tab, k, chains, steps, seed=12345, burn_in=steps // 4)
    n = tab.shape[0]
    for c in range(chains):
        assert np.array_equal(init[c], oracle.init_order(12345, c, n))
    assert np.array_equal(gpu.chains_read(ch, "trace_accept"), ref["trace_accept"])
    assert np.array_equal(gpu.chains_read(ch, "trace_score"), ref["trace_score"])
    assert np.array_equal(gpu.chains_read(ch, "orders"), ref["final_orders"])
    assert np.array_equal(gpu.chains_read(ch, "scores"), ref["final_score"])
    assert np.array_equal(gpu.chains_read(ch, "best_scores"), ref["best_score"])
    assert np.array_equal(gpu.chains_read(ch, "best_orders"), ref["best_order"])
    assert np.array_equal(gpu.chains_read(ch, "best_ranks"), ref["best_rank"])
    assert np.array_equal(gpu.chains_read(ch, "accepts"), ref["accepts"])
    assert np.array_equal(gpu.chains_read(ch, "edge_counts").astype(np.uint64), ref["edge_counts"])
    assert gpu.chains_read(ch, "steps")[0] == steps


def test_literal_log_variant(gpu):
    tab, k = _shared()
    ch, _, ref = _run_both(gpu, tab, k, 2, 300, seed=9, literal=True)
    assert np.array_equal(gpu.chains_read(ch, "trace_accept"), ref["trace_accept"])


def test_steps_in_pieces_equal_one_run(gpu):
    tab, k = _shared("n20_k4_m1000")
    t = gpu.table_from_scores(tab, k)
    a = gpu.chains_create(t, 4, 77, trace_cap=100)
    gpu.chains_step(a, 100)
    b = gpu.chains_create(t, 4, 77, trace_cap=100)
    for s in (1, 2, 30, 67):
        gpu.chains_step(b, s)
    assert np.array_equal(gpu.chains_read(a, "trace_score"), gpu.chains_read(b, "trace_score"))
    assert np.array_equal(gpu.chains_read(a, "orders"), gpu.chains_read(b, "orders"))


def test_init_orders_given(gpu):
    tab, k = _shared()
    t = gpu.table_from_scores(tab, k)
    init = synth.random_orders(6, 5, 1)
    ch = gpu.chains_create(t, 5, 4, init_orders=init, trace_cap=50)
    gpu.chains_step(ch, 50)
    ref = oracle.mcmc_run(tab, k, 5, 50, seed=4, init_orders=init, trace=True)
    assert np.array_equal(gpu.chains_read(ch, "trace_score"), ref["trace_score"])


def test_mcmc_run_outputs(gpu):
    data, arity, k, R, net = synth.workload("n20_k4_m1000")
    tab = oracle.build_table(data, arity, k, R=R)
    t = gpu.table_from_scores(tab, k)
    out = gpu.mcmc_run(t, chains=6, steps=400, seed=21, burn_in=100)
    ref = oracle.mcmc_run(tab, k, 6, 400, seed=21, burn_in=100)
    c = int(np.argmax(ref["best_score"]))
    assert out["best_score"] == ref["best_score"][c]
    assert np.array_equal(out["best_order"], ref["best_order"][c])
    assert np.array_equal(out["best_dag"], oracle.greedy_dag(20, k, ref["best_rank"][c]))
    f = ref["edge_counts"].sum(0) / (6 * 300)
    np.testing.assert_allclose(out["edge_freq"], f, rtol=0, atol=1e-15)
    # the best DAG is acyclic and consistent with the best order
    pos = np.empty(20, int)
    pos[out["best_order"]] = np.arange(20)
    ii, mm = np.nonzero(out["best_dag"])
    assert (pos[mm] < pos[ii]).all()


def test_ess_matches_oracle_on_recorded_series(gpu):
    tab, k = _shared("n6_k2_m100", 1)
    n = tab.shape[0]
    t = gpu.table_from_scores(tab, k)
    C, steps, burn = 4, 3000, 200
    ch = gpu.chains_create(t, C, 5, burn_in=burn, record_every=1, record_cap=steps)
    gpu.chains_step(ch, steps)
    T = int(gpu.chains_read(ch, "record_len")[0])
    assert T == steps - burn
    bits = gpu.chains_read(ch, "record")
    ess = gpu.chains_read(ch, "ess")
    counts = gpu.chains_read(ch, "edge_counts")
    for i in range(n):
        for m in range(n):
            tot, any_ = 0.0, False
            for c in range(C):
                words = bits[c, i, m]
                x = np.array([(int(words[t >> 6]) >> (t & 63)) & 1 for t in range(T)], np.float64)
                assert x.sum() == counts[c, i, m]          # every post-burn-in step recorded
                e = oracle.ess(x)
                if not np.isnan(e):
                    tot += e
                    any_ = True
            if any_:
                assert ess[i, m] == pytest.approx(tot, rel=1e-9)
            else:
                assert np.isnan(ess[i, m])
