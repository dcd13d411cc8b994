"""Failure detection without a GPU fault: every device-side wait in the library is
bounded; when one runs out the kernel records it and returns, and the host reports
BN_ETIMEOUT with the context still usable.  The self test waits on an mbarrier nothing
arrives at and a flag nothing sets."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_bounded_waits_time_out_and_context_survives(gpu):
    L = gpu.lib()
    L.bn_selftest_timeout.argtypes = [C.c_int64, C.c_void_p]
    rc = L.bn_selftest_timeout(50_000_000, None)          # 50 ms
    assert rc == gpu.ETIMEOUT, gpu.last_error()
    # the context still works: a normal call afterwards succeeds and is correct
    data, arity, k, R, _ = synth.workload("n6_k2_m100")
    t = gpu.build_scores(data, arity, k)
    br, sc = gpu.score_orders(t, synth.random_orders(6, 8, 1))
    assert np.isfinite(sc).all()
    assert L.bn_selftest_timeout(0, None) == gpu.EINVAL
