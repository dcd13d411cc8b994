"""bn_score_orders_noalloc, the order-scoring call for callers that cannot allocate
device memory (a memory pool that owns the device, a loop that cannot afford the
synchronisation of cudaMalloc/cudaFree, a plugin given pre-allocated buffers).  It keeps
its work lists in a static device array instead of allocating; its results must be those
of bn_score_orders: the same ranks bit for bit and the same scores.

This file is collected last so that a run stopping at its first failure has run every
other test first.  It must pass alone in a fresh process as well."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _noalloc(bn, t, orders_dev, torch):
    B, n = orders_dev.shape
    br = torch.full((B, n), -1, dtype=torch.int32, device=orders_dev.device)
    sc = torch.full((B,), float("nan"), dtype=torch.float64, device=orders_dev.device)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = bn.lib().bn_score_orders_noalloc(t.handle, C.c_void_p(orders_dev.data_ptr()), B,
                                          C.c_void_p(br.data_ptr()), C.c_void_p(sc.data_ptr()), stream)
    assert rc == bn.OK, bn.last_error()
    return br.cpu().numpy().view(np.uint32), sc.cpu().numpy()


def test_noalloc_matches_score_orders_on_two_calls(gpu):
    import torch
    bn = gpu
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    t = bn.build_scores(data, arity, k, R=R)
    # two calls in a row: a large batch, then a smaller one that must not see the first
    # call's leftovers in the shared array
    for B, seed in ((300, 1), (37, 2)):
        orders = synth.random_orders(20, B, seed)
        ref_rank, ref_score = bn.score_orders(t, orders)
        rank, score = _noalloc(bn, t, torch.as_tensor(orders, device="cuda"), torch)
        assert np.array_equal(rank, ref_rank)
        assert np.array_equal(score, ref_score)


@pytest.mark.parametrize("mode,B", [("full", 8), ("full", 97), ("full", 420), ("pruned", 64), ("unrank", 64),
                                    ("sliced", 64), ("sorted", 300)])
def test_noalloc_every_scan_path(gpu, mode, B):
    """The kernels the call can dispatch to: the scan of all nodes' rank range with up to
    eight orders a thread (n * ceil(B / 8) <= 1,024 items; B = 8 and 97 at n = 20), the
    full-table scan (B = 420), the scan over the pruned table's survivors, the scan that
    unranks parent sets on the fly and the two bit-sliced scans; two calls in a row, each
    equal to bn_score_orders on the same table and mode."""
    import torch
    bn = gpu
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    t = bn.build_scores(data, arity, k, R=R)
    bn.table_set_scan(t, {"full": bn.SCAN_FULL, "pruned": bn.SCAN_PRUNED, "unrank": bn.SCAN_UNRANK,
                          "sliced": bn.SCAN_SLICED, "sorted": bn.SCAN_SORTED}[mode])
    for seed in (5, 6):
        orders = synth.random_orders(20, B, seed)
        ref_rank, ref_score = bn.score_orders(t, orders)
        rank, score = _noalloc(bn, t, torch.as_tensor(orders, device="cuda"), torch)
        assert np.array_equal(rank, ref_rank)
        assert np.array_equal(score, ref_score)


def test_noalloc_full_size_and_limit(gpu):
    import torch
    bn = gpu
    data, arity, k, R, _ = synth.workload("n60_k4_m1000")
    t = bn.build_scores(data, arity, k, R=R)
    orders = synth.random_orders(60, 256, 3)
    ref_rank, ref_score = bn.score_orders(t, orders)
    od = torch.as_tensor(orders, device="cuda")
    for _ in range(2):
        rank, score = _noalloc(bn, t, od, torch)
        assert np.array_equal(rank, ref_rank)
        assert np.array_equal(score, ref_score)
    # a batch beyond the static array is refused with a clear error, nothing launched
    big = torch.zeros((12000, 60), dtype=torch.uint8, device="cuda")
    rc = bn.lib().bn_score_orders_noalloc(t.handle, C.c_void_p(big.data_ptr()), 12000, None, None,
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == bn.EINVAL and "scratch" in bn.last_error()
