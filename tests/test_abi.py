"""CPU-side checks of the C-ABI library: it loads, exports every symbol include/bn.h
declares, and its host-only helpers and argument checks behave (no GPU work)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bn():
    from paper_1210_5128_gb300 import build as b
    b.build()
    import paper_1210_5128_gb300 as mod
    return mod


def _declared():
    src = open(os.path.join(ROOT, "include", "bn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bn_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_abi(bn):
    decl = _declared()
    assert set(bn.ABI) <= set(decl)
    for name in decl:
        assert hasattr(bn.lib(), name), f"{name} declared in bn.h but not exported"


def test_exports_match_nm(bn):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", bn.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (bn_[a-z_0-9]+)$", out, flags=re.M))
    assert set(_declared()) <= exported


def test_version_and_error_string(bn):
    assert "sm_103a" in bn.version()
    assert isinstance(bn.last_error(), str)


@pytest.mark.parametrize("N,k", [(5, 2), (19, 4), (59, 4), (63, 3)])
def test_rank_helpers_match_oracle(bn, N, k):
    rng = np.random.default_rng(N * 10 + k)
    S = oracle.num_sets(N, k)
    for r in list(range(min(S, 50))) + list(rng.integers(0, S, 200)) + [S - 1]:
        r = int(r)
        mask = bn.unrank(N, k, r)
        assert [c for c in range(N) if mask >> c & 1] == oracle.unrank(N, k, r)
        assert bn.rank(N, k, mask) == r


def test_rank_helper_errors(bn):
    with pytest.raises(bn.BNError) as e:
        bn.unrank(5, 2, oracle.num_sets(5, 2))
    assert e.value.code == bn.EINVAL
    with pytest.raises(bn.BNError):
        bn.rank(5, 2, 0b111)          # three bits > k
    with pytest.raises(bn.BNError):
        bn.rank(5, 2, 1 << 5)         # bit at N


def test_argument_checks_before_any_device_work(bn):
    L = bn.lib()
    h = C.c_void_p()
    data = np.zeros((4, 3), np.uint8)
    ar = np.full(3, 2, np.uint8)
    # n out of range, k out of range, arity out of range, NULL out
    assert L.bn_build_scores(data.ctypes.data, 4, 1, ar.ctypes.data, 0, None, None, 0, None, C.byref(h)) == bn.EINVAL
    assert L.bn_build_scores(data.ctypes.data, 4, 65, ar.ctypes.data, 0, None, None, 0, None, C.byref(h)) == bn.EINVAL
    assert L.bn_build_scores(data.ctypes.data, 4, 3, ar.ctypes.data, 3, None, None, 0, None, C.byref(h)) == bn.EINVAL
    bad = np.array([2, 5, 2], np.uint8)
    assert L.bn_build_scores(data.ctypes.data, 4, 3, bad.ctypes.data, 1, None, None, 0, None, C.byref(h)) == bn.EINVAL
    assert "arity" in bn.last_error()
    d2 = data.copy()
    d2[2, 1] = 2
    assert L.bn_build_scores(d2.ctypes.data, 4, 3, ar.ctypes.data, 1, None, None, 0, None, C.byref(h)) == bn.EINVAL
    R = np.full((3, 3), 0.5)
    R[0, 1] = np.nan
    assert L.bn_build_scores(data.ctypes.data, 4, 3, ar.ctypes.data, 1, R.ctypes.data, None, 0, None,
                             C.byref(h)) == bn.EINVAL
    R[0, 1] = 1.5
    assert L.bn_build_scores(data.ctypes.data, 4, 3, ar.ctypes.data, 1, R.ctypes.data, None, 0, None,
                             C.byref(h)) == bn.EINVAL
    assert L.bn_build_scores(data.ctypes.data, 4, 3, ar.ctypes.data, 1, None, None, 0, None, None) == bn.EINVAL
    assert L.bn_score_orders(None, None, 1, None, None, 0, None) == bn.EINVAL
    assert L.bn_table_info(None, None, None, None, None) == bn.EINVAL


def test_argument_checks_of_batch_and_run_calls(bn):
    """The calls added for batches, runs and measurement reject bad arguments before any
    device work (the messages name the offending network)."""
    L = bn.lib()
    good = np.zeros((4, 3), np.uint8)
    bad = np.full((4, 3), 7, np.uint8)
    ar = np.full(3, 2, np.uint8)
    datas = (C.c_void_p * 2)(good.ctypes.data, bad.ctypes.data)
    ars = (C.c_void_p * 2)(ar.ctypes.data, ar.ctypes.data)
    ms, ns, ks = (C.c_int * 2)(4, 4), (C.c_int * 2)(3, 3), (C.c_int * 2)(1, 1)
    out = (C.c_void_p * 2)()
    assert L.bn_build_scores_batch(2, datas, ms, ns, ars, ks, None, None, 0, None, out) == bn.EINVAL
    assert "network 1" in bn.last_error() and out[0] is None and out[1] is None
    assert L.bn_build_scores_batch(0, datas, ms, ns, ars, ks, None, None, 0, None, out) == bn.EINVAL
    p = bn.MCMCParams(4, 0, 1, 0, 0, 0, 0, 0, 0, 0.1, 0, 0, None)
    tabs = (C.c_void_p * 1)(None)
    ps = (bn.MCMCParams * 1)(p)
    assert L.bn_mcmc_run_batch(0, tabs, ps, 10, None, None, None, None, None, None) == bn.EINVAL
    assert L.bn_mcmc_run_batch(1, tabs, ps, 10, None, None, None, None, None, None) == bn.EINVAL
    assert "network 0" in bn.last_error()
    assert L.bn_mcmc_run(None, C.byref(p), 10, None, None, None, None, None, None) == bn.EINVAL
    assert L.bn_chains_set_learned_launch(None, 0) == bn.EINVAL
    assert L.bn_measure_test_rate(None, None) == bn.EINVAL


def test_binding_constants_equal_the_header(bn):
    """Every named constant the Python binding passes through the C ABI (error codes,
    memory kinds, scan modes, output ids, proposal kinds, learned launch modes) has the
    value bn.h defines, so a call never sends one mode meaning another."""
    src = open(os.path.join(ROOT, "include", "bn.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"^#define BN_([A-Z0-9_]+)\s+(-?\d+)", src, flags=re.M)}
    checked = 0
    for name, value in defs.items():
        if name.startswith("OUT_"):
            assert bn.OUT[name[4:].lower()] == value, name
        elif name.startswith("MLP_"):
            continue                               # tensor ids: bn.MLP_TENSORS order, below
        elif hasattr(bn, name):
            assert getattr(bn, name) == value, name
        else:
            continue
        checked += 1
    assert checked >= 30
    for i, t in enumerate(bn.MLP_TENSORS):
        assert defs["MLP_" + t.upper()] == i
    for mode in ("FULL", "PRUNED", "UNRANK", "SLICED", "SORTED"):
        assert getattr(bn, "SCAN_" + mode) == defs["SCAN_" + mode]
