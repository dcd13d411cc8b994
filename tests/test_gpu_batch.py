"""Batches of networks of uneven size, n, arity, m and k: every network's chains in one
fused launch must produce exactly what stepping each network alone produces, and a
network switched to the learned proposal steps through its own path inside the batch."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

OUTS = ("trace_score", "trace_accept", "orders", "scores", "best_scores", "best_orders", "best_ranks", "accepts",
        "edge_counts", "steps", "items")


def _nets(count, seed, nmax=60):
    out = []
    rng = np.random.default_rng(seed)
    for t in range(count):
        n = int(rng.integers(6, nmax + 1))
        ar = rng.integers(2, 5, size=n).astype(np.uint8)
        m = int(rng.integers(50, 400))
        k = int(rng.integers(2, 5))
        net = synth.random_network(n, 3, ar, seed * 100 + t)
        out.append((synth.forward_sample(net, m, seed * 100 + t + 1), ar, k))
    return out


def test_batch_equals_networks_alone(gpu):
    nets = _nets(7, 3)
    assert max(d.shape[1] for d, _, _ in nets) > 33          # spans beyond one warp's lanes
    tables = []
    for data, ar, k in nets:
        t = gpu.build_scores(data, ar, k)
        gpu.table_set_scan(t, gpu.SCAN_PRUNED)
        tables.append(t)
    chains = [5, 32, 1, 17, 64, 3, 40]
    seeds = [11 * i + 1 for i in range(len(tables))]
    b = gpu.batch_create(tables, chains, seeds, burn_in=20, trace_cap=400)
    for s in (150, 250):
        b.step(s)
    for i, t in enumerate(tables):
        alone = gpu.chains_create(t, chains[i], seeds[i], burn_in=20, trace_cap=400)
        gpu.chains_step(alone, 400)
        for what in OUTS:
            assert np.array_equal(gpu.chains_read(b.chains(i), what), gpu.chains_read(alone, what)), (i, what)


def test_batch_untraced_equals_full_scan_alone(gpu):
    """The many-network launch without score traces (FP64 scores of fast-accepted moves
    left for later) against each network stepped alone on its full table, per step."""
    nets = _nets(5, 8)
    tables = []
    for data, ar, k in nets:
        t = gpu.build_scores(data, ar, k)
        gpu.table_set_scan(t, gpu.SCAN_PRUNED)
        tables.append(t)
    chains = [9, 32, 3, 20, 48]
    seeds = [7 * i + 3 for i in range(len(tables))]
    b = gpu.batch_create(tables, chains, seeds, burn_in=50)
    for s in (300, 500):
        b.step(s)
    for i, t in enumerate(tables):
        gpu.table_set_scan(t, gpu.SCAN_FULL)
        alone = gpu.chains_create(t, chains[i], seeds[i], burn_in=50)
        gpu.chains_step(alone, 800)
        for what in ("orders", "scores", "best_scores", "best_orders", "best_ranks", "accepts", "edge_counts",
                     "steps", "items"):
            assert np.array_equal(gpu.chains_read(b.chains(i), what), gpu.chains_read(alone, what)), (i, what)


def test_batch_of_many_blocks_equals_full_scan_alone(gpu):
    """More blocks than fit two per SM: the launch caps its shared-memory survivor caches so
    every block is resident, and networks above the cap run on their global-memory
    caches; every network's results still equal stepping it alone on its full table."""
    nets = _nets(20, 21)
    tables = []
    for data, ar, k in nets:
        t = gpu.build_scores(data, ar, k)
        gpu.table_set_scan(t, gpu.SCAN_PRUNED)
        tables.append(t)
    chains = [128] * len(tables)                  # 20 x 128 chains = 320 blocks of 8
    seeds = [5 * i + 2 for i in range(len(tables))]
    b = gpu.batch_create(tables, chains, seeds, burn_in=20)
    b.step(300)
    for i, t in enumerate(tables):
        gpu.table_set_scan(t, gpu.SCAN_FULL)
        alone = gpu.chains_create(t, chains[i], seeds[i], burn_in=20)
        gpu.chains_step(alone, 300)
        for what in ("orders", "scores", "best_scores", "best_orders", "best_ranks", "accepts", "edge_counts",
                     "steps", "items"):
            assert np.array_equal(gpu.chains_read(b.chains(i), what), gpu.chains_read(alone, what)), (i, what)


def test_batch_network_vs_oracle(gpu):
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    tab = oracle.build_table(data, arity, k, R=R)
    t6 = synth.workload("n6_k2_m100")
    tab6 = oracle.build_table(t6[0], t6[1], t6[2])
    ta = gpu.table_from_scores(tab, k)
    tb = gpu.table_from_scores(tab6, t6[2])
    for t in (ta, tb):
        gpu.table_set_scan(t, gpu.SCAN_PRUNED)
    b = gpu.batch_create([ta, tb], [6, 4], [77, 78], burn_in=10, trace_cap=300)
    b.step(300)
    ref = oracle.mcmc_run(tab, k, 6, 300, seed=77, burn_in=10, trace=True)
    assert np.array_equal(gpu.chains_read(b.chains(0), "trace_score"), ref["trace_score"])
    assert np.array_equal(gpu.chains_read(b.chains(0), "edge_counts").astype(np.uint64), ref["edge_counts"])
    ref6 = oracle.mcmc_run(tab6, t6[2], 4, 300, seed=78, burn_in=10, trace=True)
    assert np.array_equal(gpu.chains_read(b.chains(1), "trace_score"), ref6["trace_score"])


def test_batch_with_learned_networks_equals_networks_alone(gpu):
    """Networks switched to the learned proposal (one trained on its own chains' history
    first) step through their own path inside the batch while the others share the fused
    launch; every network's results equal stepping it alone with the same proposal."""
    nets = _nets(4, 5)
    tables = []
    for data, ar, k in nets:
        t = gpu.build_scores(data, ar, k)
        gpu.table_set_scan(t, gpu.SCAN_PRUNED)
        tables.append(t)
    chains = [16, 24, 8, 32]
    seeds = [9, 10, 11, 12]
    learned = {1: 0.2, 3: 0.1}                         # network -> eps_mix

    def weights(i):
        n = gpu.table_info(tables[i])["n"]
        return n, synth.mlp_init_weights(n, 8, 128, 2 + i)

    b = gpu.batch_create(tables, chains, seeds, burn_in=30, trace_cap=300)
    keep = []
    for i, eps in learned.items():
        n, w = weights(i)
        net = gpu.mlp_create(n, w, hidden=128, d=8, batch_cap=chains[i], lr=1e-3)
        keep.append(net)
        if i == 3:                                    # trained on its own history first
            gpu.chains_set_proposal(b.chains(i), net, gpu.PROPOSAL_TRAIN, eps_mix=eps)
            gpu.chains_step(b.chains(i), 100)
        gpu.chains_set_proposal(b.chains(i), net, gpu.PROPOSAL_LEARNED, eps_mix=eps)
    b.step(200)
    for i, t in enumerate(tables):
        alone = gpu.chains_create(t, chains[i], seeds[i], burn_in=30, trace_cap=300)
        if i in learned:
            n, w = weights(i)
            net = gpu.mlp_create(n, w, hidden=128, d=8, batch_cap=chains[i], lr=1e-3)
            keep.append(net)
            if i == 3:
                gpu.chains_set_proposal(alone, net, gpu.PROPOSAL_TRAIN, eps_mix=learned[i])
                gpu.chains_step(alone, 100)
            gpu.chains_set_proposal(alone, net, gpu.PROPOSAL_LEARNED, eps_mix=learned[i])
            gpu.chains_step(alone, 200)
        else:
            gpu.chains_step(alone, 200)
        for what in OUTS:
            assert np.array_equal(gpu.chains_read(b.chains(i), what), gpu.chains_read(alone, what)), (i, what)
        assert gpu.chains_read(b.chains(i), "accepts").max() > 0


def test_mcmc_run_batch_equals_single_runs(gpu):
    """bn_mcmc_run_batch: every network's one-shot results (best state, DAG, edge
    frequencies, acceptance and ESS) equal its own bn_mcmc_run with the same parameters,
    uniform and learned networks mixed."""
    nets = _nets(4, 13)
    tables = []
    for data, ar, k in nets:
        t = gpu.build_scores(data, ar, k)
        gpu.table_set_scan(t, gpu.SCAN_PRUNED)
        tables.append(t)
    chains, seeds = [16, 8, 32, 4], [3, 4, 5, 6]
    props = [gpu.PROPOSAL_UNIFORM, gpu.PROPOSAL_LEARNED, gpu.PROPOSAL_UNIFORM, gpu.PROPOSAL_UNIFORM]
    out = gpu.mcmc_run_batch(tables, chains, 400, seeds, burn_in=40, thin=2, proposals=props, eps_mix=0.2,
                             train_iters=60)
    for i, t in enumerate(tables):
        one = gpu.mcmc_run(t, chains[i], 400, seed=seeds[i], burn_in=40, thin=2, proposal=props[i], eps_mix=0.2,
                           train_iters=60)
        for key in ("best_order", "best_dag", "edge_freq"):
            assert np.array_equal(out[i][key], one[key]), (i, key)
        assert out[i]["best_score"] == one["best_score"]
        for key in ("acceptance", "uncertain_edges", "order_evals"):
            assert out[i]["stats"][key] == one["stats"][key], (i, key)
        a, b = out[i]["stats"]["ess_median"], one["stats"]["ess_median"]
        assert (np.isnan(a) and np.isnan(b)) or a == b
