"""Python access to the plain CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
leg are the only callers.  The CUDA library never imports or links this package.

The C library is compiled with gcc on first use (or by ``build()``) next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain -O2, no vectorisation flags)."""
    stale = force or not os.path.exists(_LIB) or \
        os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        # no FMA contraction: the same FP64 results on x86-64 and aarch64 hosts
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


_u8p = C.POINTER(C.c_uint8)
_u32p = C.POINTER(C.c_uint32)
_u64p = C.POINTER(C.c_uint64)
_i64p = C.POINTER(C.c_int64)
_ip = C.POINTER(C.c_int)
_dp = C.POINTER(C.c_double)


class MCMCParams(C.Structure):
    _fields_ = [("chains", C.c_int), ("iters", C.c_int64), ("burn_in", C.c_int64),
                ("seed", C.c_uint64), ("literal_log", C.c_int), ("chain0", C.c_int)]


def _declare(L):
    L.orc_binom.restype = C.c_uint64
    L.orc_binom.argtypes = [C.c_int, C.c_int]
    L.orc_num_sets.restype = C.c_int64
    L.orc_num_sets.argtypes = [C.c_int, C.c_int]
    L.orc_rank.restype = C.c_int64
    L.orc_rank.argtypes = [C.c_int, C.c_int, _ip, C.c_int]
    L.orc_unrank.restype = C.c_int
    L.orc_unrank.argtypes = [C.c_int, C.c_int, C.c_int64, _ip]
    L.orc_comb_alg2.restype = None
    L.orc_comb_alg2.argtypes = [C.c_int, C.c_int, C.c_int64, _ip]
    L.orc_counts.restype = None
    L.orc_counts.argtypes = [_u8p, C.c_int, C.c_int, _u8p, C.c_int, _ip, C.c_int, _u32p]
    L.orc_local_score.restype = C.c_double
    L.orc_local_score.argtypes = [_u8p, C.c_int, C.c_int, _u8p, C.c_int, _ip, C.c_int,
                                  C.c_int, C.c_double, C.c_double, _dp]
    L.orc_ppf.restype = C.c_double
    L.orc_ppf.argtypes = [C.c_double]
    L.orc_build_table_node.restype = None
    L.orc_build_table_node.argtypes = [_u8p, C.c_int, C.c_int, _u8p, C.c_int, C.c_int,
                                       C.c_double, C.c_double, _dp, C.c_int, _dp]
    L.orc_build_table.restype = None
    L.orc_build_table.argtypes = [_u8p, C.c_int, C.c_int, _u8p, C.c_int, C.c_int,
                                  C.c_double, C.c_double, _dp, _dp]
    L.orc_cand_to_node.restype = C.c_int
    L.orc_cand_to_node.argtypes = [C.c_int, C.c_int]
    L.orc_order_score.restype = C.c_double
    L.orc_order_score.argtypes = [_dp, C.c_int, C.c_int, _u8p, _u32p]
    L.orc_order_score_sum.restype = C.c_double
    L.orc_order_score_sum.argtypes = [_dp, C.c_int, C.c_int, _u8p, _dp]
    L.orc_greedy_dag.restype = None
    L.orc_greedy_dag.argtypes = [C.c_int, C.c_int, _u32p, _u8p]
    L.orc_graph_score.restype = C.c_double
    L.orc_graph_score.argtypes = [_dp, C.c_int, C.c_int, _u32p]
    L.orc_philox4x64.restype = None
    L.orc_philox4x64.argtypes = [_u64p, _u64p, _u64p]
    L.orc_mcmc_run.restype = None
    L.orc_mcmc_run.argtypes = [_dp, C.c_int, C.c_int, C.POINTER(MCMCParams), _u8p,
                               _u8p, _dp, _u8p, _dp, _u32p, _u64p, _i64p, _dp, _u8p]
    L.orc_init_order.restype = None
    L.orc_init_order.argtypes = [C.c_uint64, C.c_int, C.c_int, _u8p]
    L.orc_pair_decode.restype = None
    L.orc_pair_decode.argtypes = [C.c_int, C.c_uint64, _ip, _ip]
    L.orc_ess.restype = C.c_double
    L.orc_ess.argtypes = [_dp, C.c_int64]
    L.orc_count_dags.restype = C.c_double
    L.orc_count_dags.argtypes = [C.c_int]


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---- combinatorics -------------------------------------------------------------------
def binom(N, j):
    return int(lib().orc_binom(N, j))


def num_sets(N, k):
    return int(lib().orc_num_sets(N, k))


def rank(N, k, subset):
    s = _c(sorted(subset), np.int32) if len(subset) else np.zeros(1, np.int32)
    return int(lib().orc_rank(N, k, _p(s, _ip), len(subset)))


def unrank(N, k, r):
    out = np.zeros(max(k, 1), np.int32)
    j = lib().orc_unrank(N, k, int(r), _p(out, _ip))
    return [int(x) for x in out[:j]]


def comb_alg2(n, k, l):
    out = np.zeros(max(k, 1), np.int32)
    lib().orc_comb_alg2(n, k, int(l), _p(out, _ip))
    return [int(x) for x in out[:k]]


# ---- counts and scores ---------------------------------------------------------------
def counts(data, arity, child, parents):
    data = _c(data, np.uint8)
    arity = _c(arity, np.uint8)
    m, n = data.shape
    ps = _c(list(parents) or [0], np.int32)
    q = int(np.prod([int(arity[p]) for p in parents], dtype=np.int64)) if parents else 1
    r = int(arity[child])
    out = np.zeros(q * r, np.uint32)
    lib().orc_counts(_p(data, _u8p), m, n, _p(arity, _u8p), child, _p(ps, _ip),
                     len(parents), _p(out, _u32p))
    return out.reshape(q, r)


def local_score(data, arity, child, parents, kind=0, ess=1.0, log10_gamma=0.0, R=None):
    data = _c(data, np.uint8)
    arity = _c(arity, np.uint8)
    m, n = data.shape
    ps = _c(sorted(parents) or [0], np.int32)
    Rp = _c(R, np.float64) if R is not None else None
    return float(lib().orc_local_score(_p(data, _u8p), m, n, _p(arity, _u8p), child,
                                       _p(ps, _ip), len(parents), kind, ess, log10_gamma,
                                       _p(Rp, _dp)))


def ppf(r):
    return float(lib().orc_ppf(r))


def _threads(threads):
    """Host threads for the calls below: None = every core.  The C calls release the
    GIL, so each thread runs the unmodified single-threaded oracle on its share."""
    return max(1, threads if threads else (os.cpu_count() or 1))


def build_table(data, arity, k, kind=0, ess=1.0, log10_gamma=0.0, R=None, threads=1):
    """Every entry of the table; with threads > 1 (None = all cores) the nodes are
    built by orc_build_table_node in parallel threads (the same entries)."""
    data = _c(data, np.uint8)
    arity = _c(arity, np.uint8)
    m, n = data.shape
    S = num_sets(n - 1, k)
    out = np.zeros((n, S), np.float64)
    Rp = _c(R, np.float64) if R is not None else None
    nt = _threads(threads)
    if nt == 1:
        lib().orc_build_table(_p(data, _u8p), m, n, _p(arity, _u8p), k, kind, ess,
                              log10_gamma, _p(Rp, _dp), _p(out, _dp))
        return out
    L = lib()

    def node(i):
        L.orc_build_table_node(_p(data, _u8p), m, n, _p(arity, _u8p), k, kind, ess,
                               log10_gamma, _p(Rp, _dp), i, _p(out[i], _dp))

    with cf.ThreadPoolExecutor(max_workers=nt) as ex:
        list(ex.map(node, range(n)))
    return out


def cand_to_node(i, c):
    return c + (1 if c >= i else 0)


def parent_set(n, k, i, r):
    """Node ids of the parent set of node i with rank r."""
    return [cand_to_node(i, c) for c in unrank(n - 1, k, r)]


def order_score(table, k, order):
    table = _c(table, np.float64)
    n = table.shape[0]
    order = _c(order, np.uint8)
    br = np.zeros(n, np.uint32)
    s = lib().orc_order_score(_p(table, _dp), n, k, _p(order, _u8p), _p(br, _u32p))
    return float(s), br


def order_scores(table, k, orders, threads=None):
    """order_score of every row of ``orders`` (B x n), the rows spread over host threads
    (None = all cores); returns (B scores, B x n best ranks)."""
    table = _c(table, np.float64)
    orders = _c(orders, np.uint8)
    B, n = orders.shape
    sc = np.zeros(B, np.float64)
    br = np.zeros((B, n), np.uint32)
    L = lib()

    def one(b):
        sc[b] = L.orc_order_score(_p(table, _dp), n, k, _p(orders[b], _u8p), _p(br[b], _u32p))

    with cf.ThreadPoolExecutor(max_workers=_threads(threads)) as ex:
        list(ex.map(one, range(B)))
    return sc, br


def order_score_sum(table, k, order):
    """The sum-based order score (log10 of the summed 10^score of every consistent
    graph) and its per-node terms."""
    table = _c(table, np.float64)
    n = table.shape[0]
    order = _c(order, np.uint8)
    ns = np.zeros(n, np.float64)
    s = lib().orc_order_score_sum(_p(table, _dp), n, k, _p(order, _u8p), _p(ns, _dp))
    return float(s), ns


def greedy_dag(n, k, best_rank):
    br = _c(best_rank, np.uint32)
    adj = np.zeros((n, n), np.uint8)
    lib().orc_greedy_dag(n, k, _p(br, _u32p), _p(adj, _u8p))
    return adj


def graph_score(table, k, ranks):
    table = _c(table, np.float64)
    r = _c(ranks, np.uint32)
    return float(lib().orc_graph_score(_p(table, _dp), table.shape[0], k, _p(r, _u32p)))


# ---- RNG and sampler -----------------------------------------------------------------
def philox4x64(ctr, key):
    c = _c(ctr, np.uint64)
    kk = _c(key, np.uint64)
    out = np.zeros(4, np.uint64)
    lib().orc_philox4x64(_p(c, _u64p), _p(kk, _u64p), _p(out, _u64p))
    return out


def init_order(seed, chain, n):
    out = np.zeros(n, np.uint8)
    lib().orc_init_order(seed, chain, n, _p(out, _u8p))
    return out


def pair_decode(n, idx):
    a = C.c_int()
    b = C.c_int()
    lib().orc_pair_decode(n, idx, C.byref(a), C.byref(b))
    return a.value, b.value


def mcmc_run(table, k, chains, iters, seed, burn_in=0, init_orders=None, trace=False,
             literal_log=False, threads=1, chain0=0):
    """orc_mcmc_run of chains chain0 .. chain0 + chains - 1; with threads > 1 (None = all
    cores) the chains are split into contiguous groups run in parallel threads, each
    group one orc_mcmc_run call with its own chain0 (the same results as one call)."""
    table = _c(table, np.float64)
    n = table.shape[0]
    io = _c(init_orders, np.uint8) if init_orders is not None else None
    out = dict(
        final_orders=np.zeros((chains, n), np.uint8),
        final_score=np.zeros(chains, np.float64),
        best_order=np.zeros((chains, n), np.uint8),
        best_score=np.zeros(chains, np.float64),
        best_rank=np.zeros((chains, n), np.uint32),
        edge_counts=np.zeros((chains, n, n), np.uint64),
        accepts=np.zeros(chains, np.int64),
    )
    ts = np.zeros((chains, iters), np.float64) if trace else None
    ta = np.zeros((chains, iters), np.uint8) if trace else None
    L = lib()

    def group(lo, hi):
        if hi <= lo:
            return
        P = MCMCParams(hi - lo, iters, burn_in, seed, 1 if literal_log else 0, chain0 + lo)
        sl = lambda a: a[lo:hi] if a is not None else None      # noqa: E731 (contiguous rows)
        L.orc_mcmc_run(_p(table, _dp), n, k, C.byref(P), _p(sl(io), _u8p),
                       _p(sl(out["final_orders"]), _u8p), _p(sl(out["final_score"]), _dp),
                       _p(sl(out["best_order"]), _u8p), _p(sl(out["best_score"]), _dp),
                       _p(sl(out["best_rank"]), _u32p), _p(sl(out["edge_counts"]), _u64p),
                       _p(sl(out["accepts"]), _i64p), _p(sl(ts), _dp), _p(sl(ta), _u8p))

    nt = min(_threads(threads), max(chains, 1))
    if nt == 1:
        group(0, chains)
    else:
        cuts = [chains * g // nt for g in range(nt + 1)]
        with cf.ThreadPoolExecutor(max_workers=nt) as ex:
            list(ex.map(lambda g: group(cuts[g], cuts[g + 1]), range(nt)))
    if trace:
        out["trace_score"] = ts
        out["trace_accept"] = ta
    return out


def ess(x):
    x = _c(x, np.float64)
    return float(lib().orc_ess(_p(x, _dp), x.shape[0]))


def count_dags(n):
    return float(lib().orc_count_dags(n))


# ---- proposal network reference (fp64 on bf16-rounded weights) -----------------------
from .mlp import *  # noqa: E402,F401,F403
