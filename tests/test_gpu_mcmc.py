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


def test_mcmc_run_stats_uniform(gpu):
    """bn_mcmc_run's summary equals what the chain API reads for the same run: acceptance
    over the steps and the ESS median/min over the uncertain edges."""
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    tab = oracle.build_table(data, arity, k, R=R)
    t = gpu.table_from_scores(tab, k)
    gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    C, steps, burn = 16, 3000, 300
    out = gpu.mcmc_run(t, C, steps, seed=8, burn_in=burn, thin=2)
    st = out["stats"]
    ch = gpu.chains_create(t, C, 8, burn_in=burn, record_every=2, record_cap=(steps - burn + 1) // 2)
    gpu.chains_step(ch, steps)
    acc = gpu.chains_read(ch, "accepts")
    assert st["acceptance"] == acc.sum() / (C * steps)
    f = gpu.chains_read(ch, "edge_counts").sum(0) / (C * (steps - burn))
    np.testing.assert_array_equal(out["edge_freq"], f)
    ess = gpu.chains_read(ch, "ess")
    unc = (f >= 0.05) & (f <= 0.95) & ~np.isnan(ess)
    assert st["uncertain_edges"] == unc.sum() > 0
    assert st["ess_median"] == np.median(ess[unc]) and st["ess_min"] == ess[unc].min()
    assert st["order_evals"] == C * steps and st["sample_ms"] > 0 and st["train_ms"] == 0
    s_ref, r_ref = oracle.order_score(tab, k, out["best_order"])
    assert out["best_score"] == s_ref
    assert np.array_equal(out["best_dag"], oracle.greedy_dag(20, k, r_ref))


def test_mcmc_run_learned_proposal(gpu):
    """The learned sampler through the one-shot call: train_iters training steps, then
    the learned proposal; the same run through the chain API gives the same results."""
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    tab = oracle.build_table(data, arity, k, R=R)
    t = gpu.table_from_scores(tab, k)
    gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    C, train, steps, burn = 32, 200, 600, 100
    w = synth.mlp_init_weights(20, 8, 128, 4)
    net_a = gpu.mlp_create(20, w, hidden=128, d=8, batch_cap=C, lr=1e-3)
    out = gpu.mcmc_run(t, C, steps, seed=9, burn_in=burn, proposal=gpu.PROPOSAL_LEARNED, eps_mix=0.2,
                       train_iters=train, thin=1, net=net_a)
    st = out["stats"]
    assert 0 < st["acceptance"] < 1 and st["order_evals"] == C * (train + steps)
    assert st["train_ms"] > 0 and st["sample_ms"] > 0
    net_b = gpu.mlp_create(20, w, hidden=128, d=8, batch_cap=C, lr=1e-3)
    ch = gpu.chains_create(t, C, 9, burn_in=burn)
    gpu.chains_set_proposal(ch, net_b, gpu.PROPOSAL_TRAIN, eps_mix=0.2)
    gpu.chains_step(ch, train)
    gpu.chains_set_proposal(ch, net_b, gpu.PROPOSAL_LEARNED, eps_mix=0.2)
    a0 = gpu.chains_read(ch, "accepts").copy()
    gpu.chains_step(ch, steps)
    f = gpu.chains_read(ch, "edge_counts").sum(0) / (C * (train + steps - burn))
    np.testing.assert_array_equal(out["edge_freq"], f)
    assert st["acceptance"] == (gpu.chains_read(ch, "accepts") - a0).sum() / (C * steps)
    c = int(np.argmax(gpu.chains_read(ch, "best_scores")))
    assert out["best_score"] == gpu.chains_read(ch, "best_scores")[c]
    s_ref, r_ref = oracle.order_score(tab, k, out["best_order"])
    assert out["best_score"] == s_ref
    assert np.array_equal(out["best_dag"], oracle.greedy_dag(20, k, r_ref))
    # the network the call creates itself (d = 32, H = 512)
    out2 = gpu.mcmc_run(t, C, 200, seed=10, proposal=gpu.PROPOSAL_LEARNED, eps_mix=0.1, train_iters=100, thin=1)
    assert out2["stats"]["order_evals"] == C * 300 and 0 < out2["stats"]["acceptance"] < 1
    with pytest.raises(gpu.BNError):
        gpu.mcmc_run(t, C, 10, seed=1, proposal=7)
    with pytest.raises(gpu.BNError):
        gpu.mcmc_run(t, C, 10, seed=1, proposal=gpu.PROPOSAL_LEARNED, eps_mix=0.0)
