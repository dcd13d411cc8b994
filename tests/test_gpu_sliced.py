"""The bit-sliced scans (BN_SCAN_SLICED: every entry, orders tested 32 at a time against
entries in score order; BN_SCAN_SORTED: the same, stopping early) must give the oracle's
order scores of Eq. (6): chosen parent-set ranks bit-exact with ties to the lowest rank,
FP64 sums identical on a shared table -- and so exactly the results of the mask-test
scan (BN_SCAN_FULL) on every table, batch size and sampler step."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

MODES = ["sliced", "sorted"]


def _mode(gpu, name):
    return {"sliced": gpu.SCAN_SLICED, "sorted": gpu.SCAN_SORTED, "full": gpu.SCAN_FULL}[name]


def _check_shared(gpu, tab, k, orders, mode):
    t = gpu.table_from_scores(tab, k)
    gpu.table_set_scan(t, _mode(gpu, mode))
    br, sc = gpu.score_orders(t, orders)
    for b, o in enumerate(orders):
        s_ref, r_ref = oracle.order_score(tab, k, o)
        assert np.array_equal(br[b], r_ref), (b, br[b], r_ref)
        assert sc[b] == s_ref
    t.free()
    return br, sc


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("B", [1, 2, 31, 32, 33, 64, 65, 129, 256, 257, 300, 1400])
def test_shared_table_n6(gpu, mode, B):
    """Ragged and whole groups of 32 orders, one to eight groups a block (B <= 256) and
    several blocks of groups per node (B > 256)."""
    data, arity, k, R, _ = synth.workload("n6_k2_m100")
    tab = oracle.build_table(data, arity, k, R=R)
    _check_shared(gpu, tab, k, synth.random_orders(6, B, 70 + B), mode)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("B", [1, 9, 97, 409])
def test_shared_table_n20_prior(gpu, mode, B):
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    tab = oracle.build_table(data, arity, k, R=R)
    _check_shared(gpu, tab, k, synth.random_orders(20, B, 90 + B), mode)


@pytest.mark.parametrize("mode", MODES)
def test_all_720_orders_n6(gpu, mode):
    import itertools
    data, arity, k, R, _ = synth.workload("n6_k2_m100", 3)
    tab = oracle.build_table(data, arity, k)
    orders = np.array(list(itertools.permutations(range(6))), np.uint8)
    _check_shared(gpu, tab, k, orders, mode)


@pytest.mark.parametrize("mode", MODES)
def test_ties_lowest_rank(gpu, mode):
    """A table of zeros: the empty set (rank 0) is the first entry in score order, so
    every node takes it; integer scores with many exact ties: the lowest tied rank."""
    n, k = 9, 3
    S = oracle.num_sets(n - 1, k)
    br, _ = _check_shared(gpu, np.zeros((n, S)), k, synth.random_orders(n, 40, 1), mode)
    assert (br == 0).all()
    rng = np.random.default_rng(0)
    tab = rng.integers(-3, 1, size=(n, S)).astype(np.float64)
    _check_shared(gpu, tab, k, synth.random_orders(n, 300, 2), mode)
    _check_shared(gpu, tab, k, synth.random_orders(n, 5, 3), mode)


@pytest.mark.parametrize("mode", MODES)
def test_empty_set_best_everywhere_and_nowhere(gpu, mode):
    """Entries beyond the empty set's sorted position are never read in the sorted mode:
    a table whose empty set beats every other set (each node takes it in every order) and
    one where it is the worst entry of its node (the cut removes nothing)."""
    n, k = 12, 4
    S = oracle.num_sets(n - 1, k)
    rng = np.random.default_rng(4)
    tab = -rng.random((n, S)) - 1.0
    tab[:, 0] = 0.0
    br, _ = _check_shared(gpu, tab, k, synth.random_orders(n, 70, 5), mode)
    assert (br == 0).all()
    tab[:, 0] = -5.0
    _check_shared(gpu, tab, k, synth.random_orders(n, 70, 6), mode)


def test_identity_and_reverse_orders(gpu):
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    tab = oracle.build_table(data, arity, k, R=R)
    o = np.arange(20, dtype=np.uint8)
    for mode in MODES:
        br, _ = _check_shared(gpu, tab, k, np.stack([o, o[::-1]]), mode)
        assert br[0, 0] == 0 and br[1, 19] == 0


@pytest.mark.parametrize("name,batches", [("n40_k4_m2000", (1, 33, 512)), ("n60_k4_m1000", (1, 4, 64, 256, 1024))])
def test_full_size_equals_mask_scan(gpu, name, batches):
    """The full-size tables the bench scores: every batch size gives the mask-test scan's
    ranks and scores bit for bit in both sliced modes, and a seeded sample of orders is
    re-scored by the oracle on the downloaded table."""
    data, arity, k, R, _ = synth.workload(name)
    n = data.shape[1]
    t = gpu.build_scores(data, arity, k, R=R)
    tab = gpu.table_scores(t)
    rng = np.random.default_rng(8)
    for B in batches:
        orders = synth.random_orders(n, B, 21 + B)
        gpu.table_set_scan(t, gpu.SCAN_FULL)
        br0, sc0 = gpu.score_orders(t, orders)
        for mode in MODES:
            gpu.table_set_scan(t, _mode(gpu, mode))
            br, sc = gpu.score_orders(t, orders)
            assert np.array_equal(br, br0), (mode, B)
            assert np.array_equal(sc, sc0), (mode, B)
        for b in sorted(set([0, B - 1] + list(rng.integers(0, B, 2)))):
            s_ref, r_ref = oracle.order_score(tab, k, orders[b])
            assert np.array_equal(br0[b], r_ref)
            assert sc0[b] == s_ref
    t.free()


@pytest.mark.parametrize("mode", MODES)
def test_sampler_steps_equal_mask_scan(gpu, mode):
    """The sampler's full-table step (work lists of the re-scored nodes of every chain):
    the same trajectories, best states and edge counts as with the mask-test scan."""
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    t = gpu.build_scores(data, arity, k, R=R)
    kw = dict(burn_in=20, trace_cap=300)
    a = gpu.chains_create(t, 40, 31, **kw)
    gpu.chains_step(a, 300)
    gpu.table_set_scan(t, _mode(gpu, mode))
    b = gpu.chains_create(t, 40, 31, **kw)
    gpu.chains_step(b, 120)
    gpu.chains_step(b, 180)
    for what in ["orders", "ranks", "scores", "best_scores", "best_orders", "best_ranks", "accepts", "edge_counts",
                 "trace_score", "trace_accept"]:
        assert np.array_equal(gpu.chains_read(a, what), gpu.chains_read(b, what)), what


def test_sliced_modes_need_k_at_most_4(gpu):
    data, arity, _, R, _ = synth.workload("n6_k2_m100")
    t = gpu.build_scores(data, arity, 5)
    for mode in MODES:
        with pytest.raises(gpu.BNError) as e:
            gpu.table_set_scan(t, _mode(gpu, mode))
        assert e.value.code == gpu.EUNSUPPORTED
    # the mask-test scan still serves the table
    orders = synth.random_orders(6, 10, 1)
    tab = gpu.table_scores(t)
    br, sc = gpu.score_orders(t, orders)
    for b, o in enumerate(orders):
        s_ref, r_ref = oracle.order_score(tab, 5, o)
        assert np.array_equal(br[b], r_ref) and sc[b] == s_ref


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,k,B", [(2, 1, 5), (3, 0, 7), (64, 2, 70), (64, 3, 33)])
def test_smallest_and_largest_networks(gpu, mode, n, k, B):
    """Edge sizes of the byte-per-parent layout: two nodes, no parents at all (k = 0, the
    empty set only), and 64 nodes, whose ids run up to 63 next to the "no parent" and
    "never" rows (64, 65); seeded random tables with exact ties."""
    rng = np.random.default_rng(n * 100 + k)
    S = oracle.num_sets(n - 1, k)
    tab = rng.integers(-40, 1, size=(n, S)).astype(np.float64) / 4.0
    _check_shared(gpu, tab, k, synth.random_orders(n, B, 7 + n), mode)


@pytest.mark.parametrize("mode", MODES)
def test_oracle_built_n60_table(gpu, oracle_n60, mode):
    """The oracle's own n = 60 table (29.4 M entries, built on the host) scored on the GPU
    in the bench's batch shape: every order's ranks and FP64 sum equal the mask-test
    scan's, and a sample equals the oracle's own order scores."""
    data, arity, k, R, tab = oracle_n60
    n = data.shape[1]
    t = gpu.table_from_scores(tab, k)
    orders = synth.random_orders(n, 97, 61)
    br0, sc0 = gpu.score_orders(t, orders)
    gpu.table_set_scan(t, _mode(gpu, mode))
    br, sc = gpu.score_orders(t, orders)
    assert np.array_equal(br, br0) and np.array_equal(sc, sc0)
    for b in (0, 31, 32, 96):
        s_ref, r_ref = oracle.order_score(tab, k, orders[b])
        assert np.array_equal(br[b], r_ref)
        assert sc[b] == s_ref
    t.free()
