"""GPU parity of the table build (counting + local score + prior) against the oracle.

Bar: every entry within 1e-12 relative (the oracle sums FP64 lgamma terms in a
canonical order, the kernel sums the same terms exactly in fixed point; both round the
same Eq. (4) expression, so their difference is a few ulp of the lgamma terms)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
RTOL = 1e-12


def _cmp(gpu, ref, atol=1e-12):
    np.testing.assert_allclose(gpu, ref, rtol=RTOL, atol=atol)


@pytest.mark.parametrize("kind,ess,lg", [(0, 1.0, 0.0), (1, 1.0, 0.0), (1, 10.0, -1.0), (0, 1.0, -0.5)])
def test_table_every_entry_n6(gpu, kind, ess, lg):
    data, arity, k, R, _ = synth.workload("n6_k2_m100")
    t = gpu.build_scores(data, arity, k, R=R, score_kind=kind, ess=ess, log10_gamma=lg)
    _cmp(gpu.table_scores(t), oracle.build_table(data, arity, k, kind, ess, lg, R))


def test_table_every_entry_n20_with_prior(gpu):
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    assert R is not None and (R != 0.5).any()
    t = gpu.build_scores(data, arity, k, R=R)
    _cmp(gpu.table_scores(t), oracle.build_table(data, arity, k, R=R))


@pytest.mark.parametrize("k", [3, 4])
@pytest.mark.parametrize("m", [0, 1, 15, 16, 17, 333])
def test_table_ragged_rows_and_mixed_arity(gpu, m, k):
    # m around the 16-row word (rows past m are zero and come out of cell 0); at k = 4 the
    # count tables reach 4 * 4 * 4 * 3 * 3 = 576 cells, so entries above 256 cells take the
    # 16-bit lanes and the rest the byte lanes in the same launch
    rng = np.random.default_rng(m)
    arity = np.array([2, 3, 4, 2, 4, 3, 2], np.uint8)
    data = np.stack([rng.integers(0, a, m) for a in arity], 1).astype(np.uint8).reshape(m, 7)
    for kind in (0, 1):
        t = gpu.build_scores(data, arity, k, score_kind=kind, ess=2.5, log10_gamma=-0.25)
        _cmp(gpu.table_scores(t), oracle.build_table(data, arity, k, kind, 2.5, -0.25))


@pytest.mark.parametrize("k", [0, 1, 5])
def test_table_degenerate_k(gpu, k):
    data, arity, _, _, _ = synth.workload("n6_k2_m100", 4)
    t = gpu.build_scores(data, arity, k)
    assert gpu.table_info(t)["sets_per_node"] == oracle.num_sets(5, k)
    _cmp(gpu.table_scores(t), oracle.build_table(data, arity, k))


def test_table_binary_large_k(gpu):
    # k = 8 with binary nodes: 512-cell count tables, 2-level template
    net = synth.random_network(10, 3, 2, 77)
    data = synth.forward_sample(net, 200, 78)
    t = gpu.build_scores(data, net.arity, 8)
    _cmp(gpu.table_scores(t), oracle.build_table(data, net.arity, 8))


def test_table_device_inputs(gpu):
    import torch
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    dd = torch.as_tensor(data, device="cuda")
    t = gpu.build_scores(dd, torch.as_tensor(arity, device="cuda"), k, R=torch.as_tensor(R, device="cuda"))
    th = gpu.build_scores(data, arity, k, R=R)
    assert np.array_equal(gpu.table_scores(t), gpu.table_scores(th))
    out = gpu.table_scores(t, device="cuda")
    assert out.is_cuda and np.array_equal(out.cpu().numpy(), gpu.table_scores(th))


def test_permuted_counts_tie_exactly(gpu):
    # relabelling a parent's states permutes the count table: the kernel's exact
    # fixed-point sum gives bit-identical entries, as the oracle's canonical sum does
    rng = np.random.default_rng(3)
    arity = np.array([3, 3, 2, 3], np.uint8)
    data = np.stack([rng.integers(0, a, 500) for a in arity], 1).astype(np.uint8)
    d2 = data.copy()
    d2[:, 1] = np.array([2, 0, 1], np.uint8)[data[:, 1]]
    a = gpu.table_scores(gpu.build_scores(data, arity, 2))
    b = gpu.table_scores(gpu.build_scores(d2, arity, 2))
    # entries of node 0 whose parent set contains node 1 are permuted tables
    assert np.array_equal(a[0], b[0])


@pytest.mark.parametrize("name", ["n40_k4_m2000", "n60_k4_m1000"])
def test_table_sampled_entries_full_size(gpu, name):
    """Full-size tables: a seeded sample of entries recomputed one by one by the
    oracle, plus the ranks at the size-class boundaries and the last rank."""
    data, arity, k, R, _ = synth.workload(name)
    n = data.shape[1]
    t = gpu.build_scores(data, arity, k, R=R)
    S = oracle.num_sets(n - 1, k)
    assert gpu.table_info(t)["sets_per_node"] == S
    rng = np.random.default_rng(17)
    edges = [0, 1, n - 2, n - 1, oracle.num_sets(n - 1, 1), oracle.num_sets(n - 1, 2),
             oracle.num_sets(n - 1, 3) - 1, S - 1]
    for i in [0, n // 2, n - 1]:
        row = gpu.table_scores(t, node=i)
        ranks = edges + list(rng.integers(0, S, 60))
        for r in ranks:
            ref = oracle.local_score(data, arity, i, oracle.parent_set(n, k, i, int(r)), R=R)
            assert abs(row[int(r)] - ref) <= RTOL * abs(ref) + 1e-12, (i, r, row[int(r)], ref)


def test_bad_data_value_on_device_rejected(gpu):
    import torch
    data = torch.zeros((20, 3), dtype=torch.uint8, device="cuda")
    data[7, 2] = 3
    with pytest.raises(gpu.BNError) as e:
        gpu.build_scores(data, np.array([2, 2, 3], np.uint8), 1)
    assert e.value.code == gpu.EINVAL


def test_batch_build_equals_single_builds(gpu):
    """bn_build_scores_batch (builds on concurrent streams) gives each network the table
    bn_build_scores gives it, entry for entry, with sorted positions that score orders the
    same; the smallest network is pinned to the oracle; a bad network is named."""
    nets = synth.uneven_batch(10, 0xB4E5_0B0B)
    tabs = gpu.build_scores_batch([(d, a, k, R) for d, a, k, R, _ in nets])
    for (d, a, k, R, _), t in zip(nets, tabs):
        single = gpu.build_scores(d, a, k, R=R)
        assert np.array_equal(gpu.table_scores(t), gpu.table_scores(single))
        orders = synth.random_orders(d.shape[1], 40, 3)
        r1, s1 = gpu.score_orders(t, orders)
        r2, s2 = gpu.score_orders(single, orders)
        assert np.array_equal(r1, r2) and np.array_equal(s1, s2)
    i = int(np.argmin([d.shape[1] for d, *_ in nets]))
    d, a, k, R, _ = nets[i]
    _cmp(gpu.table_scores(tabs[i]), oracle.build_table(d, a, k, R=R, threads=None))
    bad = [(nets[0][0], nets[0][1], nets[0][2], None),
           (np.full((5, 3), 7, np.uint8), np.array([2, 2, 2], np.uint8), 1, None)]
    with pytest.raises(gpu.BNError) as e:
        gpu.build_scores_batch(bad)
    assert e.value.code == gpu.EINVAL and "network 1" in str(e.value)


def test_profiled_build_equals_build(gpu):
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    t0 = gpu.build_scores(data, arity, k, R=R)
    t1, ms = gpu.build_scores_profiled(data, arity, k, R=R)
    assert ms > 0.0
    assert np.array_equal(gpu.table_scores(t0), gpu.table_scores(t1))
