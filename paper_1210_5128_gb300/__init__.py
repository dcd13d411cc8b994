"""Python binding of libbngpu.so, the GB300 order-space Bayesian-network scorer.

Argument marshalling only: every step runs in the library's CUDA kernels behind the C
ABI declared in include/bn.h, and the names here are the C names without the ``bn_``
prefix.  Arrays may be numpy arrays / CPU tensors (host memory, results come back as
numpy arrays) or CUDA tensors (device memory, results are CUDA tensors on the same
device and the call runs on torch's current stream).

There is no CPU fallback: if the shared library is missing or cannot be loaded the
import fails with the reason.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbngpu.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = 0, -1, -2, -3, -4, -5
MEM_HOST, MEM_DEVICE = 0, 1
OUT = dict(orders=1, scores=2, ranks=3, best_orders=4, best_scores=5, best_ranks=6,
           edge_counts=7, accepts=8, trace_score=9, trace_accept=10, steps=11, ess=12, record=13,
           record_len=14, items=15, logits=16)

# names the ABI exports (include/bn.h); tests check the library against this list
ABI = ["bn_build_scores", "bn_table_from_scores", "bn_table_info", "bn_table_scores",
       "bn_table_free", "bn_score_orders", "bn_unrank", "bn_rank", "bn_chains_create",
       "bn_chains_step", "bn_chains_step_profiled", "bn_chains_read", "bn_chains_free",
       "bn_mcmc_run", "bn_last_error", "bn_version", "bn_kernel_launches"]


class BNError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class ScoreParams(C.Structure):
    _fields_ = [("score_kind", C.c_int), ("ess", C.c_double), ("log10_gamma", C.c_double)]


class MCMCParams(C.Structure):
    _fields_ = [("chains", C.c_int), ("burn_in", C.c_int64), ("seed", C.c_uint64),
                ("literal_log", C.c_int), ("record_every", C.c_int), ("record_cap", C.c_int),
                ("trace", C.c_int), ("trace_cap", C.c_int64),
                ("proposal", C.c_int), ("eps_mix", C.c_double), ("train_iters", C.c_int64),
                ("thin", C.c_int), ("net", C.c_void_p)]


class MCMCStats(C.Structure):
    _fields_ = [("acceptance", C.c_double), ("ess_median", C.c_double), ("ess_min", C.c_double),
                ("uncertain_edges", C.c_int64), ("sample_ms", C.c_double), ("train_ms", C.c_double),
                ("order_evals", C.c_int64)]


class MLPParams(C.Structure):
    _fields_ = [("d", C.c_int), ("hidden", C.c_int), ("batch_cap", C.c_int), ("lr", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("adam_eps", C.c_float)]


MLP_TENSORS = ["E", "W1", "b1", "W2", "b2", "W3", "b3"]

_vp = C.c_void_p
_L = None


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libbngpu.so is not built ({LIB_PATH}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    _L = C.CDLL(LIB_PATH)
    _L.bn_last_error.restype = C.c_char_p
    _L.bn_version.restype = C.c_char_p
    _L.bn_kernel_launches.restype = C.c_int64
    _L.bn_build_scores.argtypes = [_vp, C.c_int, C.c_int, _vp, C.c_int, _vp, C.POINTER(ScoreParams),
                                   C.c_int, _vp, C.POINTER(_vp)]
    _L.bn_table_from_scores.argtypes = [_vp, C.c_int, C.c_int, C.c_int, _vp, C.POINTER(_vp)]
    _L.bn_build_scores_profiled.argtypes = [_vp, C.c_int, C.c_int, _vp, C.c_int, _vp, C.POINTER(ScoreParams),
                                            C.c_int, _vp, C.POINTER(_vp), C.POINTER(C.c_double)]
    _L.bn_build_scores_batch.argtypes = [C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_int, _vp, _vp]
    _L.bn_table_info.argtypes = [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int64),
                                 C.POINTER(C.c_int64)]
    _L.bn_table_scores.argtypes = [_vp, C.c_int, _vp, C.c_int, _vp]
    _L.bn_table_free.argtypes = [_vp]
    _L.bn_table_free.restype = None
    _L.bn_score_orders.argtypes = [_vp, _vp, C.c_int, _vp, _vp, C.c_int, _vp]
    _L.bn_score_orders_noalloc.argtypes = [_vp, _vp, C.c_int, _vp, _vp, _vp]
    _L.bn_score_orders_profiled.argtypes = [_vp, _vp, C.c_int, _vp, _vp, C.c_int, _vp, C.POINTER(C.c_double)]
    _L.bn_score_orders_sum.argtypes = [_vp, _vp, C.c_int, _vp, _vp, C.c_int, _vp]
    _L.bn_unrank.argtypes = [C.c_int, C.c_int, C.c_int64, C.POINTER(C.c_uint64)]
    _L.bn_rank.argtypes = [C.c_int, C.c_int, C.c_uint64, C.POINTER(C.c_int64)]
    _L.bn_chains_create.argtypes = [_vp, C.POINTER(MCMCParams), _vp, C.c_int, _vp, C.POINTER(_vp)]
    _L.bn_chains_step.argtypes = [_vp, C.c_int64, _vp]
    _L.bn_chains_step_profiled.argtypes = [_vp, C.c_int64, _vp, C.POINTER(C.c_double),
                                               C.POINTER(C.c_int64)]
    _L.bn_chains_read.argtypes = [_vp, C.c_int, _vp, C.c_int, _vp]
    _L.bn_chains_free.argtypes = [_vp]
    _L.bn_chains_free.restype = None
    _L.bn_mcmc_run.argtypes = [_vp, C.POINTER(MCMCParams), C.c_int64, _vp, _vp, _vp, _vp,
                               C.POINTER(MCMCStats), _vp]
    _L.bn_mcmc_run_batch.argtypes = [C.c_int, _vp, _vp, C.c_int64, _vp, _vp, _vp, _vp, _vp, _vp]
    _L.bn_measure_test_rate.argtypes = [_vp, C.POINTER(C.c_double)]
    _L.bn_chains_set_learned_launch.argtypes = [_vp, C.c_int]
    _L.bn_mlp_create.argtypes = [C.c_int, C.POINTER(MLPParams)] + [_vp] * 7 + [C.c_int, _vp, C.POINTER(_vp)]
    _L.bn_mlp_forward.argtypes = [_vp, _vp, C.c_int, _vp, C.c_int, _vp]
    _L.bn_mlp_loss_grad.argtypes = [_vp, _vp, _vp, _vp, C.c_int, _vp, C.c_int, _vp]
    _L.bn_mlp_adam_step.argtypes = [_vp, _vp]
    _L.bn_mlp_read.argtypes = [_vp, C.c_int, _vp, C.c_int, _vp]
    _L.bn_mlp_free.argtypes = [_vp]
    _L.bn_mlp_free.restype = None
    _L.bn_gemm_bf16.argtypes = [_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, _vp]
    _L.bn_chains_set_proposal.argtypes = [_vp, _vp, C.c_int, C.c_double, _vp]
    _L.bn_table_set_scan.argtypes = [_vp, C.c_int, _vp]
    _L.bn_table_pruned.argtypes = [_vp, _vp]
    _L.bn_table_autotune.argtypes = [_vp, C.c_int, _vp, _vp]
    _L.bn_batch_create.argtypes = [C.c_int, _vp, _vp, _vp, C.POINTER(_vp)]
    _L.bn_batch_chains.argtypes = [_vp, C.c_int, C.POINTER(_vp)]
    _L.bn_batch_step.argtypes = [_vp, C.c_int64, _vp]
    _L.bn_batch_free.argtypes = [_vp]
    _L.bn_batch_free.restype = None
    _L.bn_selftest_timeout.argtypes = [C.c_int64, _vp]
    return _L


def lib():
    """The loaded C library (loaded on first use; raises if it is not built)."""
    global _L
    if _L is None:
        _L = _load()
    return _L


def last_error() -> str:
    return lib().bn_last_error().decode()


def version() -> str:
    return lib().bn_version().decode()


def kernel_launches() -> int:
    return int(lib().bn_kernel_launches())


def _check(rc):
    if rc != OK:
        raise BNError(rc, last_error())


# ---- marshalling ---------------------------------------------------------------------
def _is_cuda(x):
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _stream(dev_tensor):
    if dev_tensor is None:
        return None
    import torch
    return C.c_void_p(torch.cuda.current_stream(dev_tensor.device).cuda_stream)


def _host(x, dtype):
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(x, dtype=dtype)


def _dev(x, tdtype):
    if x.dtype != tdtype:
        x = x.to(tdtype)
    return x.contiguous()


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


class Table:
    """Owns a bn_table*; freed with the object (or explicitly with free())."""

    def __init__(self, handle):
        self._h = handle

    @property
    def handle(self):
        if not self._h:
            raise ValueError("table already freed")
        return self._h

    def free(self):
        if self._h:
            lib().bn_table_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self):
        return table_info(self)


def build_scores(data, arity, k, R=None, score_kind=0, ess=1.0, log10_gamma=0.0) -> Table:
    """Local-score table of Eq. (4) + prior of Eq. (9) (bn_build_scores)."""
    p = ScoreParams(score_kind, ess, log10_gamma)
    h = _vp()
    if _is_cuda(data):
        import torch
        d = _dev(data, torch.uint8)
        a = _dev(arity.to(d.device) if hasattr(arity, "to") else torch.as_tensor(np.asarray(arity, np.uint8),
                                                                                 device=d.device), torch.uint8)
        r = None
        if R is not None:
            r = _dev(R.to(d.device) if hasattr(R, "to") else torch.as_tensor(np.asarray(R, np.float64),
                                                                             device=d.device), torch.float64)
        m, n = d.shape
        _check(lib().bn_build_scores(_ptr(d), m, n, _ptr(a), k, _ptr(r), C.byref(p), MEM_DEVICE,
                                  _stream(d), C.byref(h)))
    else:
        d = _host(data, np.uint8)
        if d.ndim != 2:
            raise ValueError("data must be (m, n)")
        a = _host(arity, np.uint8)
        r = _host(R, np.float64) if R is not None else None
        m, n = d.shape
        _check(lib().bn_build_scores(_ptr(d), m, n, _ptr(a), k, _ptr(r), C.byref(p), MEM_HOST,
                                  None, C.byref(h)))
    return Table(h)


def build_scores_profiled(data, arity, k, R=None, score_kind=0, ess=1.0, log10_gamma=0.0):
    """bn_build_scores_profiled on host arrays: (table, device ms of the build kernel)."""
    p = ScoreParams(score_kind, ess, log10_gamma)
    h = _vp()
    d = _host(data, np.uint8)
    a = _host(arity, np.uint8)
    r = _host(R, np.float64) if R is not None else None
    m, n = d.shape
    ms = C.c_double()
    _check(lib().bn_build_scores_profiled(_ptr(d), m, n, _ptr(a), k, _ptr(r), C.byref(p), MEM_HOST, None,
                                          C.byref(h), C.byref(ms)))
    return Table(h), ms.value


def build_scores_batch(nets, score_kind=0, ess=1.0, log10_gamma=0.0):
    """bn_build_scores_batch: one table per (data, arity, k, R) of ``nets`` (R may be None),
    host arrays, built concurrently."""
    cnt = len(nets)
    keep = []
    dps, aps, rps = (C.c_void_p * cnt)(), (C.c_void_p * cnt)(), (C.c_void_p * cnt)()
    ms, ns, ks = (C.c_int * cnt)(), (C.c_int * cnt)(), (C.c_int * cnt)()
    for i, (data, arity, k, R) in enumerate(nets):
        d = _host(data, np.uint8)
        a = _host(arity, np.uint8)
        r = _host(R, np.float64) if R is not None else None
        keep += [d, a, r]
        dps[i] = d.ctypes.data
        aps[i] = a.ctypes.data
        rps[i] = r.ctypes.data if r is not None else None
        ms[i], ns[i], ks[i] = d.shape[0], d.shape[1], int(k)
    prm = (ScoreParams * cnt)(*[ScoreParams(score_kind, ess, log10_gamma) for _ in range(cnt)])
    out = (C.c_void_p * cnt)()
    _check(lib().bn_build_scores_batch(cnt, dps, ms, ns, aps, ks, rps, prm, MEM_HOST, None, out))
    return [Table(C.c_void_p(out[i])) for i in range(cnt)]


def table_from_scores(scores, k) -> Table:
    h = _vp()
    if _is_cuda(scores):
        import torch
        s = _dev(scores, torch.float64)
        _check(lib().bn_table_from_scores(_ptr(s), s.shape[0], k, MEM_DEVICE, _stream(s), C.byref(h)))
    else:
        s = _host(scores, np.float64)
        _check(lib().bn_table_from_scores(_ptr(s), s.shape[0], k, MEM_HOST, None, C.byref(h)))
    return Table(h)


def table_info(t: Table):
    n, k, S, b = C.c_int(), C.c_int(), C.c_int64(), C.c_int64()
    _check(lib().bn_table_info(t.handle, C.byref(n), C.byref(k), C.byref(S), C.byref(b)))
    return dict(n=n.value, k=k.value, sets_per_node=S.value, device_bytes=b.value)


def table_scores(t: Table, node: int = -1, device=None):
    info = table_info(t)
    rows = info["n"] if node < 0 else 1
    shape = (rows, info["sets_per_node"]) if node < 0 else (info["sets_per_node"],)
    if device is not None:
        import torch
        out = torch.empty(shape, dtype=torch.float64, device=device)
        _check(lib().bn_table_scores(t.handle, node, _ptr(out), MEM_DEVICE, _stream(out)))
        return out
    out = np.empty(shape, np.float64)
    _check(lib().bn_table_scores(t.handle, node, _ptr(out), MEM_HOST, None))
    return out


def score_orders(t: Table, orders):
    """Eq. (6) for a batch of orders (bn_score_orders) -> (best_rank (B,n), score (B,))."""
    n = table_info(t)["n"]
    if _is_cuda(orders):
        import torch
        o = _dev(orders, torch.uint8)
        B = o.shape[0]
        br = torch.empty((B, n), dtype=torch.int32, device=o.device)
        sc = torch.empty((B,), dtype=torch.float64, device=o.device)
        _check(lib().bn_score_orders(t.handle, _ptr(o), B, _ptr(br), _ptr(sc), MEM_DEVICE, _stream(o)))
        return br, sc
    o = _host(orders, np.uint8).reshape(-1, n)
    B = o.shape[0]
    br = np.empty((B, n), np.uint32)
    sc = np.empty((B,), np.float64)
    _check(lib().bn_score_orders(t.handle, _ptr(o), B, _ptr(br), _ptr(sc), MEM_HOST, None))
    return br, sc


def score_orders_profiled(t: Table, orders):
    """score_orders on device tensors with the scan kernel's device time (ms, CUDA events
    around its launch): (best_rank, score, scan_ms)."""
    import torch
    n = table_info(t)["n"]
    o = _dev(orders, torch.uint8)
    B = o.shape[0]
    br = torch.empty((B, n), dtype=torch.int32, device=o.device)
    sc = torch.empty((B,), dtype=torch.float64, device=o.device)
    ms = C.c_double()
    _check(lib().bn_score_orders_profiled(t.handle, _ptr(o), B, _ptr(br), _ptr(sc), MEM_DEVICE, _stream(o),
                                          C.byref(ms)))
    return br, sc, ms.value


def score_orders_sum(t: Table, orders):
    """The sum-based order score (bn_score_orders_sum) -> (order score (B,), node terms (B, n));
    device tensors in, device tensors out; host arrays in, numpy arrays out."""
    n = table_info(t)["n"]
    if _is_cuda(orders):
        import torch
        o = _dev(orders, torch.uint8)
        B = o.shape[0]
        sc = torch.empty((B,), dtype=torch.float64, device=o.device)
        ns = torch.empty((B, n), dtype=torch.float64, device=o.device)
        _check(lib().bn_score_orders_sum(t.handle, _ptr(o), B, _ptr(sc), _ptr(ns), MEM_DEVICE, _stream(o)))
        return sc, ns
    o = _host(orders, np.uint8).reshape(-1, n)
    B = o.shape[0]
    sc = np.empty((B,), np.float64)
    ns = np.empty((B, n), np.float64)
    _check(lib().bn_score_orders_sum(t.handle, _ptr(o), B, _ptr(sc), _ptr(ns), MEM_HOST, None))
    return sc, ns


SCAN_FULL, SCAN_PRUNED, SCAN_UNRANK, SCAN_SLICED, SCAN_SORTED = 0, 1, 2, 3, 4


def table_set_scan(t: Table, mode: int):
    """Scan mode of a table (bn_table_set_scan): SCAN_FULL, SCAN_PRUNED, SCAN_UNRANK,
    SCAN_SLICED or SCAN_SORTED."""
    _check(lib().bn_table_set_scan(t.handle, mode, None))


def table_autotune(t: Table, max_items: int):
    """Time the full scan's tilings and keep the fastest -> (stage size, blocks per node,
    microseconds per launch)."""
    out = np.zeros(3, np.int64)
    _check(lib().bn_table_autotune(t.handle, max_items, None, _ptr(out)))
    return tuple(int(x) for x in out)


def table_pruned(t: Table):
    """Surviving entries per node after pruning."""
    out = np.zeros(table_info(t)["n"], np.int64)
    _check(lib().bn_table_pruned(t.handle, _ptr(out)))
    return out


def measure_test_rate(stream=None) -> float:
    """Measured peak of the scan's consistency test on this GPU, tests per second
    (bn_measure_test_rate)."""
    r = C.c_double()
    _check(lib().bn_measure_test_rate(stream, C.byref(r)))
    return r.value


def unrank(N, k, rank) -> int:
    m = C.c_uint64()
    _check(lib().bn_unrank(N, k, rank, C.byref(m)))
    return m.value


def rank(N, k, mask) -> int:
    r = C.c_int64()
    _check(lib().bn_rank(N, k, mask, C.byref(r)))
    return r.value


# ---- sampler -------------------------------------------------------------------------
class Chains:
    def __init__(self, handle, table, n, params):
        self._h = handle
        self.table = table          # keeps the table alive
        self.n = n
        self.params = params

    @property
    def handle(self):
        if not self._h:
            raise ValueError("chains already freed")
        return self._h

    def free(self):
        if self._h:
            lib().bn_chains_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def chains_create(t: Table, chains, seed, burn_in=0, init_orders=None, literal_log=False,
                  record_every=0, record_cap=0, trace_cap=0) -> Chains:
    n = table_info(t)["n"]
    p = MCMCParams(chains, burn_in, seed, 1 if literal_log else 0, record_every, record_cap,
                   1 if trace_cap else 0, trace_cap, 0, 0.0, 0, 0, None)
    h = _vp()
    io = _host(init_orders, np.uint8) if init_orders is not None else None
    _check(lib().bn_chains_create(t.handle, C.byref(p), _ptr(io), MEM_HOST, None, C.byref(h)))
    return Chains(h, t, n, p)


def chains_step(c: Chains, steps: int, stream=None):
    _check(lib().bn_chains_step(c.handle, steps, stream))


def chains_step_profiled(c: Chains, steps: int, stream=None):
    """Returns (summed scan-kernel ms, scan launches) measured with CUDA events."""
    ms, nl = C.c_double(), C.c_int64()
    _check(lib().bn_chains_step_profiled(c.handle, steps, stream, C.byref(ms), C.byref(nl)))
    return ms.value, nl.value


_OUT_SHAPES = {
    "orders": (np.uint8, "cn"), "scores": (np.float64, "c"), "ranks": (np.uint32, "cn"),
    "best_orders": (np.uint8, "cn"), "best_scores": (np.float64, "c"),
    "best_ranks": (np.uint32, "cn"), "edge_counts": (np.uint32, "cnn"),
    "accepts": (np.int64, "c"), "trace_score": (np.float64, "ct"),
    "trace_accept": (np.uint8, "ct"), "steps": (np.int64, "1"), "ess": (np.float64, "nn"),
    "record": (np.uint64, "cnnw"), "record_len": (np.int64, "1"), "items": (np.int64, "1"),
    "logits": (np.float32, "cP"),
}


def chains_read(c: Chains, what: str):
    dtype, dims = _OUT_SHAPES[what]
    size = {"c": c.params.chains, "n": c.n, "t": c.params.trace_cap, "1": 1, "P": c.n * (c.n - 1) // 2,
            "w": max(1, (c.params.record_cap + 63) // 64) if c.params.record_every > 0 else 0}
    shape = tuple(size[d] for d in dims)
    out = np.empty(shape, dtype)
    _check(lib().bn_chains_read(c.handle, OUT[what], _ptr(out), MEM_HOST, None))
    return out


def mcmc_run(t: Table, chains, steps, seed, burn_in=0, literal_log=False, proposal=0, eps_mix=0.1,
             train_iters=0, thin=0, net=None):
    """Algorithm 1 end to end (bn_mcmc_run): best order, its greedy DAG, best score, edge
    frequencies and the run's summary (acceptance, edge-posterior ESS when thin > 0,
    device times).  proposal = PROPOSAL_LEARNED trains the network (given, or one the
    call creates) for train_iters steps first."""
    n = table_info(t)["n"]
    p = MCMCParams(chains, burn_in, seed, 1 if literal_log else 0, 0, 0, 0, 0,
                   proposal, eps_mix, train_iters, thin, net.handle if net is not None else None)
    bo = np.empty(n, np.uint8)
    dag = np.empty((n, n), np.uint8)
    bs = np.empty(1, np.float64)
    ef = np.empty((n, n), np.float64)
    st = MCMCStats()
    _check(lib().bn_mcmc_run(t.handle, C.byref(p), steps, _ptr(bo), _ptr(dag), _ptr(bs), _ptr(ef), C.byref(st),
                             None))
    stats = {f: getattr(st, f) for f, _ in MCMCStats._fields_}
    return dict(best_order=bo, best_dag=dag, best_score=float(bs[0]), edge_freq=ef, stats=stats)


def mcmc_run_batch(tables, chains, steps, seeds, burn_in=0, thin=0, proposals=None, eps_mix=0.1,
                   train_iters=0):
    """bn_mcmc_run_batch: one-shot runs of many networks stepped together; ``chains`` and
    ``seeds`` are ints or per-network lists, ``proposals`` None (uniform) or a list.
    Returns one dict per network, as mcmc_run."""
    cnt = len(tables)
    chains = chains if hasattr(chains, "__len__") else [chains] * cnt
    seeds = seeds if hasattr(seeds, "__len__") else [seeds + i for i in range(cnt)]
    proposals = proposals or [PROPOSAL_UNIFORM] * cnt
    ps = (MCMCParams * cnt)(*[MCMCParams(int(chains[i]), burn_in, int(seeds[i]), 0, 0, 0, 0, 0, int(proposals[i]),
                                         eps_mix, train_iters, thin, None) for i in range(cnt)])
    hs = (C.c_void_p * cnt)(*[t.handle for t in tables])
    ns = [table_info(t)["n"] for t in tables]
    bo = [np.empty(n, np.uint8) for n in ns]
    dag = [np.empty((n, n), np.uint8) for n in ns]
    ef = [np.empty((n, n), np.float64) for n in ns]
    bs = np.empty(cnt, np.float64)
    st = (MCMCStats * cnt)()
    ptrs = lambda arrs: (C.c_void_p * cnt)(*[a.ctypes.data for a in arrs])      # noqa: E731
    _check(lib().bn_mcmc_run_batch(cnt, hs, ps, steps, ptrs(bo), ptrs(dag), _ptr(bs), ptrs(ef), st, None))
    return [dict(best_order=bo[i], best_dag=dag[i], best_score=float(bs[i]), edge_freq=ef[i],
                 stats={f: getattr(st[i], f) for f, _ in MCMCStats._fields_}) for i in range(cnt)]


# ---- learned proposal ----------------------------------------------------------------
class MLP:
    """Owns a bn_mlp* (the learned swap proposal network)."""

    def __init__(self, handle, n, d, hidden, cap):
        self._h, self.n, self.d, self.hidden, self.cap = handle, n, d, hidden, cap
        self.P = n * (n - 1) // 2

    @property
    def handle(self):
        if not self._h:
            raise ValueError("network already freed")
        return self._h

    def free(self):
        if self._h:
            lib().bn_mlp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def mlp_create(n, weights, hidden=512, d=32, batch_cap=256, lr=1e-3) -> MLP:
    """weights: dict E, W1, b1, W2, b2, W3, b3 (float arrays, unpadded row-major)."""
    p = MLPParams(d, hidden, batch_cap, lr, 0.0, 0.0, 0.0)
    ws = [_host(weights[k], np.float32) for k in MLP_TENSORS]
    h = _vp()
    _check(lib().bn_mlp_create(n, C.byref(p), *[_ptr(w) for w in ws], MEM_HOST, None, C.byref(h)))
    return MLP(h, n, d, hidden, batch_cap)


def mlp_forward(m: MLP, orders):
    o = _host(orders, np.uint8).reshape(-1, m.n)
    out = np.empty((o.shape[0], m.P), np.float32)
    _check(lib().bn_mlp_forward(m.handle, _ptr(o), o.shape[0], _ptr(out), MEM_HOST, None))
    return out


def mlp_loss_grad(m: MLP, orders, pairs, alpha):
    o = _host(orders, np.uint8).reshape(-1, m.n)
    pr = _host(pairs, np.uint32)
    al = _host(alpha, np.float32)
    loss = np.zeros(1, np.float32)
    _check(lib().bn_mlp_loss_grad(m.handle, _ptr(o), _ptr(pr), _ptr(al), o.shape[0], _ptr(loss), MEM_HOST, None))
    return float(loss[0])


def mlp_adam_step(m: MLP):
    _check(lib().bn_mlp_adam_step(m.handle, None))


def mlp_read(m: MLP, name: str, grad=False):
    shapes = {"E": (m.n, m.d), "W1": (m.hidden, m.n * m.d), "b1": (m.hidden,), "W2": (m.hidden, m.hidden),
              "b2": (m.hidden,), "W3": (m.P, m.hidden), "b3": (m.P,)}
    out = np.empty(shapes[name], np.float32)
    what = MLP_TENSORS.index(name) + (7 if grad else 0)
    _check(lib().bn_mlp_read(m.handle, what, _ptr(out), MEM_HOST, None))
    return out


class _BorrowedChains(Chains):
    """Chains owned by a batch (freed with it)."""

    def free(self):
        self._h = None


class Batch:
    """Owns a bn_batch*: many networks' chains stepped together (bn_batch_*)."""

    def __init__(self, handle, tables, chains_list):
        self._h, self.tables, self._chains = handle, tables, chains_list

    def chains(self, i) -> Chains:
        return self._chains[i]

    def step(self, steps, stream=None):
        _check(lib().bn_batch_step(self._h, steps, stream))

    def free(self):
        if self._h:
            lib().bn_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def batch_create(tables, chains, seeds, burn_in=0, record_every=0, record_cap=0, trace_cap=0) -> Batch:
    """One chain set per table; `chains` and `seeds` are ints or per-network lists."""
    cnt = len(tables)
    chains = chains if hasattr(chains, "__len__") else [chains] * cnt
    seeds = seeds if hasattr(seeds, "__len__") else [seeds + i for i in range(cnt)]
    ps = (MCMCParams * cnt)(*[MCMCParams(int(chains[i]), burn_in, int(seeds[i]), 0, record_every, record_cap,
                                         1 if trace_cap else 0, trace_cap) for i in range(cnt)])
    hs = (C.c_void_p * cnt)(*[t.handle for t in tables])
    h = _vp()
    _check(lib().bn_batch_create(cnt, hs, ps, None, C.byref(h)))
    lst = []
    for i in range(cnt):
        ch = _vp()
        _check(lib().bn_batch_chains(h, i, C.byref(ch)))
        lst.append(_BorrowedChains(ch, tables[i], table_info(tables[i])["n"], ps[i]))
    return Batch(h, tables, lst)


PROPOSAL_UNIFORM, PROPOSAL_LEARNED, PROPOSAL_TRAIN = 0, 1, 2


def chains_set_proposal(c: Chains, mlp, mode, eps_mix=0.1, stream=None):
    """Proposal of the chains' next steps (bn_chains_set_proposal)."""
    c.mlp = mlp                 # keeps the network alive with the chains
    _check(lib().bn_chains_set_proposal(c.handle, mlp.handle if mlp is not None else None, mode, eps_mix,
                                        stream))


LEARNED_LAUNCH_AUTO, LEARNED_LAUNCH_GRAPH = 0, 1


def chains_set_learned_launch(c: Chains, mode):
    """Persistent cooperative launch (AUTO, when it fits) or three kernels per step from a
    CUDA graph (GRAPH) for the learned proposal; the results are the same."""
    _check(lib().bn_chains_set_learned_launch(c.handle, mode))


def gemm_bf16(A, B):
    """C = A @ B.T on the tensor cores; A (M, K), B (N, K) bf16 CUDA tensors."""
    import torch
    assert A.is_cuda and A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16
    A, B = A.contiguous(), B.contiguous()
    M, K = A.shape
    N = B.shape[0]
    out = torch.empty((M, N), dtype=torch.float32, device=A.device)
    _check(lib().bn_gemm_bf16(_ptr(A), _ptr(B), _ptr(out), M, N, K, _stream(A)))
    return out
