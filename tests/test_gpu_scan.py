"""GPU parity of the order score (Eq. 6): chosen parent-set ranks bit-exact (ties to the
lowest rank) and order scores within 1e-9 relative -- exact on a shared table, where
both sides add the same FP64 entries in ascending node id."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _check_shared(gpu, tab, k, orders, mode=None):
    t = gpu.table_from_scores(tab, k)
    if mode is not None:
        gpu.table_set_scan(t, mode)
    br, sc = gpu.score_orders(t, orders)
    for b, o in enumerate(orders):
        s_ref, r_ref = oracle.order_score(tab, k, o)
        assert np.array_equal(br[b], r_ref), (b, br[b], r_ref)
        assert sc[b] == s_ref
    return br, sc


@pytest.mark.parametrize("B", [1, 2, 3, 5, 8, 17, 31, 33, 37, 256, 300, 1400])
def test_shared_table_n6(gpu, B):
    data, arity, k, R, _ = synth.workload("n6_k2_m100")
    tab = oracle.build_table(data, arity, k, R=R)
    _check_shared(gpu, tab, k, synth.random_orders(6, B, B))


@pytest.mark.parametrize("B", [1, 3, 9, 16, 51, 97, 409])
def test_shared_table_n20_prior(gpu, B):
    """Every dispatch of bn_score_orders: the scan of all nodes' rank range with R orders
    a thread and T threads per (node, order group) item -- (T, R) = (8, 1), (8, 3), (4, 5),
    (4, 8), (1, 8) in 256-thread blocks, (1, 8) with 260 items (a ragged last warp) -- and
    the full-table scan once n * ceil(B / 8) exceeds 1,024 items (B = 409)."""
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    tab = oracle.build_table(data, arity, k, R=R)
    _check_shared(gpu, tab, k, synth.random_orders(20, B, 4 + B))


def test_profiled_scoring_equals_plain(gpu):
    import torch
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    t = gpu.build_scores(data, arity, k, R=R)
    for B in (1, 7, 300):
        orders = synth.random_orders(20, B, 40 + B)
        br, sc = gpu.score_orders(t, orders)
        br2, sc2, ms = gpu.score_orders_profiled(t, torch.as_tensor(orders, device="cuda"))
        assert np.array_equal(br, br2.cpu().numpy().astype(np.uint32))
        assert np.array_equal(sc, sc2.cpu().numpy())
        assert ms > 0.0


def test_all_720_orders_n6(gpu):
    import itertools
    data, arity, k, R, _ = synth.workload("n6_k2_m100", 2)
    tab = oracle.build_table(data, arity, k)
    orders = np.array(list(itertools.permutations(range(6))), np.uint8)
    br, sc = _check_shared(gpu, tab, k, orders)
    assert sc.max() == max(oracle.order_score(tab, k, o)[0] for o in orders)


def test_ties_lowest_rank(gpu):
    n, k = 9, 3
    S = oracle.num_sets(n - 1, k)
    tab = np.zeros((n, S))
    br, sc = _check_shared(gpu, tab, k, synth.random_orders(n, 40, 1))
    assert (br == 0).all()
    rng = np.random.default_rng(0)
    tab = rng.integers(-3, 1, size=(n, S)).astype(np.float64)   # many exact ties
    _check_shared(gpu, tab, k, synth.random_orders(n, 300, 2))
    _check_shared(gpu, tab, k, synth.random_orders(n, 5, 3))


def test_identity_and_reverse_orders(gpu):
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    tab = oracle.build_table(data, arity, k, R=R)
    o = np.arange(20, dtype=np.uint8)
    br, _ = _check_shared(gpu, tab, k, np.stack([o, o[::-1]]))
    assert br[0, 0] == 0 and br[1, 19] == 0          # the first node takes the empty set


def test_end_to_end_independent_tables_n20(gpu):
    """GPU table + GPU scan vs oracle table + oracle scan: indices must agree; a
    disagreement is only acceptable between two entries within 1e-12 of each other."""
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    ref_tab = oracle.build_table(data, arity, k, R=R)
    t = gpu.build_scores(data, arity, k, R=R)
    orders = synth.random_orders(20, 128, 9)
    br, sc = gpu.score_orders(t, orders)
    near = 0
    for b, o in enumerate(orders):
        s_ref, r_ref = oracle.order_score(ref_tab, k, o)
        assert abs(sc[b] - s_ref) <= 1e-9 * abs(s_ref)
        for i in np.nonzero(br[b] != r_ref)[0]:
            a, c = ref_tab[i, br[b][i]], ref_tab[i, r_ref[i]]
            assert abs(a - c) <= 1e-12 * abs(c)
            near += 1
    assert near == 0


def test_device_tensors(gpu):
    import torch
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    t = gpu.build_scores(data, arity, k, R=R)
    orders = synth.random_orders(20, 64, 3)
    br_h, sc_h = gpu.score_orders(t, orders)
    br_d, sc_d = gpu.score_orders(t, torch.as_tensor(orders, device="cuda"))
    assert np.array_equal(br_d.cpu().numpy().astype(np.uint32), br_h)
    assert np.array_equal(sc_d.cpu().numpy(), sc_h)


def test_empty_batch_and_bad_orders(gpu):
    data, arity, k, R, _ = synth.workload("n6_k2_m100")
    t = gpu.build_scores(data, arity, k)
    br, sc = gpu.score_orders(t, np.zeros((0, 6), np.uint8))
    assert br.shape == (0, 6) and sc.shape == (0,)
    bad = np.array([[0, 1, 2, 3, 4, 4]], np.uint8)
    with pytest.raises(gpu.BNError) as e:
        gpu.score_orders(t, bad)
    assert e.value.code == gpu.EINVAL
    bad = np.array([[0, 1, 2, 3, 4, 9]], np.uint8)
    with pytest.raises(gpu.BNError):
        gpu.score_orders(t, bad)


def test_autotuned_tiling_gives_identical_results(gpu):
    data, arity, k, R, _ = synth.workload("n40_k4_m2000")
    t = gpu.build_scores(data, arity, k, R=R)
    orders = synth.random_orders(40, 256, 12)
    br0, sc0 = gpu.score_orders(t, orders)
    sub, nchunk, us = gpu.table_autotune(t, 256)
    assert sub in (512, 1024, 2048) and nchunk >= 1 and us > 0
    br1, sc1 = gpu.score_orders(t, orders)
    assert np.array_equal(br0, br1) and np.array_equal(sc0, sc1)


@pytest.mark.parametrize("name,B", [("n40_k4_m2000", 512), ("n60_k4_m1000", 256), ("n60_k4_m1000", 4)])
def test_full_size_sampled_orders(gpu, name, B):
    """The full-size table built on the GPU, scored in the bench's batch shape; a seeded
    sample of the orders is re-scored by the oracle on the downloaded table."""
    data, arity, k, R, _ = synth.workload(name)
    n = data.shape[1]
    t = gpu.build_scores(data, arity, k, R=R)
    tab = gpu.table_scores(t)
    orders = synth.random_orders(n, B, 11)
    br, sc = gpu.score_orders(t, orders)
    rng = np.random.default_rng(5)
    for b in sorted(set([0, B - 1] + list(rng.integers(0, B, 4)))):
        s_ref, r_ref = oracle.order_score(tab, k, orders[b])
        assert np.array_equal(br[b], r_ref)
        assert sc[b] == s_ref
    # invariants on every order: the first node takes the empty set, and every score is
    # the sum of its chosen entries
    for b in range(B):
        assert br[b][orders[b][0]] == 0
    picked = tab[np.arange(n)[None, :], br.astype(np.int64)]
    np.testing.assert_allclose(picked.sum(1), sc, rtol=1e-12)


@pytest.mark.parametrize("name,B", [("n6_k2_m100", 37), ("n20_k4_m1000", 300), ("n40_k4_m2000", 256),
                                    ("n60_k4_m1000", 64)])
def test_unranked_parent_sets_equal_the_table(gpu, name, B):
    """BN_SCAN_UNRANK computes every parent set from its rank inside the scan (no table
    read); ranks and scores must equal the table-driven scan bit for bit."""
    data, arity, k, R, _ = synth.workload(name)
    n = data.shape[1]
    t = gpu.build_scores(data, arity, k, R=R)
    orders = synth.random_orders(n, B, 77)
    br_f, sc_f = gpu.score_orders(t, orders)
    gpu.table_set_scan(t, gpu.SCAN_UNRANK)
    br_u, sc_u = gpu.score_orders(t, orders)
    assert np.array_equal(br_f, br_u)
    assert np.array_equal(sc_f, sc_u)


@pytest.mark.parametrize("name,B", [("n6_k2_m100", 37), ("n20_k4_m1000", 5), ("n20_k4_m1000", 300)])
def test_unranked_parent_sets_against_oracle(gpu, name, B):
    """BN_SCAN_UNRANK (Algorithm 2's strategy: every parent set computed from its index
    in the scan) on the oracle's table against the oracle's brute-force order score."""
    data, arity, k, R, _ = synth.workload(name)
    tab = oracle.build_table(data, arity, k, R=R)
    _check_shared(gpu, tab, k, synth.random_orders(data.shape[1], B, 55 + B), mode=gpu.SCAN_UNRANK)


def test_unranked_n40_against_oracle(gpu, oracle_n40):
    """The unranked scan on the oracle's table of the 40-node workload (k = 4)."""
    _, _, k, _, tab = oracle_n40
    t = gpu.table_from_scores(tab, k)
    gpu.table_set_scan(t, gpu.SCAN_UNRANK)
    orders = synth.random_orders(40, 64, 4)
    br, sc = gpu.score_orders(t, orders)
    sc_ref, br_ref = oracle.order_scores(tab, k, orders[:16])
    assert np.array_equal(br[:16], br_ref) and np.array_equal(sc[:16], sc_ref)


def test_unranked_sampler_equals_table_sampler(gpu):
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    t = gpu.build_scores(data, arity, k, R=R)
    a = gpu.chains_create(t, 32, 12, trace_cap=150)
    gpu.chains_step(a, 150)
    gpu.table_set_scan(t, gpu.SCAN_UNRANK)
    b = gpu.chains_create(t, 32, 12, trace_cap=150)
    gpu.chains_step(b, 150)
    for what in ("trace_score", "orders", "ranks", "best_scores", "edge_counts"):
        assert np.array_equal(gpu.chains_read(a, what), gpu.chains_read(b, what)), what
