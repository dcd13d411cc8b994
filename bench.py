#!/usr/bin/env python
"""Throughput of the order-space MH sampler (Algorithm 1) on one GB300.

An MH iteration of a chain: a swap proposal, the order score of Eq. (6) of the proposed
order (an exact full-order score; only the nodes between the swapped positions are
re-scored, the others keep their best sets), the MH test, best-graph and edge-count
updates.  A timed step is --iters-per-step (default 1,000) iterations of every chain.
Workload: 60 ternary nodes, in-degree <= 3, m = 1000 synthetic samples, k = 4 (489,406
parent sets per node, 29.36 M FP64 entries, 235 MB), 256 chains.

The headline runs the pruned table (only entries that no subset of their parent set
matches or beats -- the same results, see include/bn.h) in the fused sampler, one launch
per timed step; the full-table scan (three kernels per iteration, replayed from a CUDA
graph) is timed beside it with its own roofline, in the mask-test and the two bit-sliced
scan modes, and bn_score_orders is swept over batch sizes in each mode.  Edge-posterior ESS/s of the plain uniform-swap
sampler and of the learned-proposal sampler (trained on the plain sampler's history) are
measured on the same table.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank runs its own replica of the
table and its own chains (independent chains, no data exchange); the value is the sum
over ranks of order evaluations divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "n60_k4_m1000"
METRIC = "order evals/s & edge-posterior ESS/s at n=60,k=4 vs plain sampler, same GB300"
UNIT = "order evals/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chains", type=int, default=256)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--iters-per-step", type=int, default=1000,
                    help="MH iterations of every chain in one timed step")
    ap.add_argument("--ess-steps", type=int, default=40000)
    ap.add_argument("--ess-thin", type=int, default=10)
    ap.add_argument("--train-steps", type=int, default=400)
    ap.add_argument("--no-ess", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the uneven 96-network batch")
    ap.add_argument("--batch-iters", type=int, default=2048)
    ap.add_argument("--batch-ess-steps", type=int, default=4000)
    ap.add_argument("--batch-train", type=int, default=300)
    ap.add_argument("--no-accuracy", action="store_true", help="skip the ROC and noise study")
    ap.add_argument("--no-configs", action="store_true", help="skip the n=20 and n=40 configurations")
    return ap.parse_args()


# ---------------------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "25"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append(dict(sm=float(p[1]), smax=float(p[2]), power=float(p[3]), hw=p[5], hwt=p[6],
                                 swt=p[7], swp=p[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(r["power"] for r in rows)}


# ---------------------------------------------------------------------------------------
# oracle (CPU) timing: reference arm and cpu_baseline
# ---------------------------------------------------------------------------------------
def _standin_table():
    """A seeded stand-in table of the workload's shape (n = 60, k = 4) for the oracle's
    timing: the oracle's order scoring enumerates the same subsets and does the same
    lookups whatever the entries' values, so its speed is that of the real table."""
    import oracle
    n, k = 60, 4
    rng = np.random.Generator(np.random.PCG64(0xB4E50003))
    return rng.standard_normal((n, oracle.num_sets(n - 1, k))) * 10.0 - 500.0, k


def oracle_sample(seconds, threads=1):
    """The oracle's sampler (Algorithm 1: a full order score per iteration) at n = 60,
    k = 4, run in short chains until ``seconds`` have passed; with threads > 1 the chains
    of a round run in parallel host threads (each the unmodified single-threaded oracle).
    Returns (order evaluations/s, evaluations, seconds, threads)."""
    import oracle
    tab, k = _standin_table()
    done, c, t0 = 0, 0, time.perf_counter()
    while True:
        oracle.mcmc_run(tab, k, threads, 4, seed=1000, chain0=c, threads=threads)
        done += 5 * threads       # per chain: the initial order + 4 proposals
        c += threads
        el = time.perf_counter() - t0
        if el >= seconds:
            return done / el, done, el, threads


def run_reference(args):
    """Reference arm: the oracle as it stands on the host's cores.  One step = one order
    evaluation (Eq. 6 by the oracle's brute-force subset walk) per host thread, each thread
    running the unmodified single-threaded oracle on its own random order of the n = 60,
    k = 4 workload."""
    import oracle
    import synth
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    tab, k = _standin_table()
    nt = os.cpu_count() or 1
    orders = synth.random_orders(60, (args.steps + 2) * nt, 4242)
    for i in range(min(args.warmup, 1)):
        oracle.order_scores(tab, k, orders[:nt], threads=nt)
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle.order_scores(tab, k, orders[(i + 1) * nt:(i + 2) * nt], threads=nt)
    tot = time.perf_counter() - t0
    value = args.steps * nt / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": run_config(args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle",
                         "sample": f"{args.steps * nt} order evaluations ({tot:.1f} s) by the oracle at n=60, "
                                   f"k=4, {nt} per step (one per host thread), on a seeded stand-in table of "
                                   "the workload's shape"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_config(args):
    """The config both arms print (the same workload and unit of work)."""
    return dict(config_dict(args.chains), iters_per_step=args.iters_per_step,
                step=f"{args.iters_per_step} MH iterations of every chain")


def config_dict(chains, scan="pruned"):
    return {"workload": f"{WORKLOAD}: 60 ternary nodes, random DAG in-degree<=3, m=1000 synthetic samples, "
                        f"k=4 (489,406 parent sets/node, 29.36M FP64 entries, 235 MB), {chains} chains, "
                        "uniform swap proposal",
            "chains": chains, "n": 60, "k": 4, "m": 1000, "scan": scan,
            "l2": "flushed: a 512 MB buffer is written and another read before every timed step (outside "
                  "its events); "
                  "the table is 235 MB of FP64 entries, the full scan streams 117 MB of sorted positions "
                  "plus the 3.9 MB mask table per pass"}


L2_FLUSH_BYTES = 512 << 20 # written, then another buffer read, between timed steps (L2 is 129 MB)
SCORE_B = (1, 2, 4, 8, 16, 32, 64, 128, 256, 1024)   # orders per bn_score_orders call in the scoring sweep
SLICED_B = (1, 4, 16, 32, 64, 128, 256, 1024, 4096)  # the same for the bit-sliced scans
ROOF_SLICED_B = 32         # the batched full-table pass of roofline_hbm: one 32-order word per node
ISSUE_PER_SM = 4           # warp schedulers per SM, one warp instruction per clock each
# ncu smsp__inst_executed.sum of k_chain_spec<1> at this workload (256 chains, 1,000-step
# launches; all four warps of a chain, the dropped speculative evaluations included), per
# chain per committed MH iteration; and dram__bytes_read.sum + dram__bytes_write.sum per
# launch of the full-table k_scan<1024,0> (256 items per node, the sampler's step)
FUSED_INST_PER_CHAIN_STEP = 760.0
FUSED_TRAFFIC_BYTES = 2.146e6    # ncu dram bytes read + written per 1,000-step launch of k_chain_spec<1>
BUILD_INST_PER_ENTRY = 649.0     # ncu smsp__inst_executed.sum of k_build<4,1,0> per entry at n=60, m=1000
SCAN_TRAFFIC_BYTES = 121.5e6
NODES_TRAFFIC_BYTES = 124.2e6    # ncu dram bytes read + written per launch of k_scan_nodes at one order
SLICED_TRAFFIC_BYTES = 120.37e6  # ncu dram bytes read + written per launch of k_scan_sliced<1,0> at 32 orders


def _flush_l2(torch, flush, stream):
    """Overwrite L2: write one buffer larger than L2, then read another, so that the timed
    kernel finds clean lines (no write-back of the flush inside the timed region)."""
    with torch.cuda.stream(stream):
        flush[0].add_(1)
        flush[1].sum()


def _timed(bn, torch, chains, steps, stream, pieces=1, flush=None):
    """Device time (ms) of `steps` MH steps run as `pieces` calls, each bracketed by CUDA
    events on the launching stream; with `flush`, L2 is flushed before every piece,
    outside the events."""
    total = 0.0
    done = 0
    for p in range(pieces):
        k = (steps - done) // (pieces - p)
        if flush is not None:
            _flush_l2(torch, flush, stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        bn.chains_step(chains, k, stream=stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
        done += k
    return total


def _accuracy(bn, synth, seed):
    """The accuracy study of Sec. VI: ROC points (TP rate, FP rate of the best graph's
    directed edges) of the 20-node workload learned prior-free and with the paper's prior
    schedule built from the prior-free run's errors, at 1,000 and 10,000 iterations of one
    chain; and the noise study: binary 20-node data with every value flipped with
    probability p, 10,000 iterations."""
    from paper_1210_5128_gb300 import roc

    def learn(data, arity, k, R, iters, s):
        t = bn.build_scores(data, arity, k, R=R)
        bn.table_set_scan(t, bn.SCAN_PRUNED)
        dag = bn.mcmc_run(t, 1, iters, seed=s, burn_in=iters // 10)["best_dag"]
        t.free()
        return dag

    data, arity, k, _, net = synth.workload("n20_k4_m1000")
    T = roc.true_adjacency(net)
    schedule = [(0.7, 0.2, 0.2), (0.7, 0.2, 0.4), (0.8, 0.1, 0.2), (0.8, 0.1, 0.4)]
    roc_pts = {}
    for iters in (1000, 10000):
        L = learn(data, arity, k, None, iters, seed)
        pts = [dict(prior="none", tp=roc.tp_fp(L, T)[0], fp=roc.tp_fp(L, T)[1])]
        for q, (rm, ra, prob) in enumerate(schedule):
            Rp = roc.prior_from_errors(L, T, rm, ra, prob, seed=seed + q)
            tp, fp = roc.tp_fp(learn(data, arity, k, Rp, iters, seed), T)
            pts.append(dict(prior=f"{rm}/{ra} p={prob}", tp=tp, fp=fp))
        roc_pts[str(iters)] = pts
    netb = synth.random_network(20, 3, 2, 0xB4E5_0A0A)
    datab = synth.forward_sample(netb, 1000, 0xB4E5_0A0B)
    Tb = roc.true_adjacency(netb)
    ar = np.full(20, 2, np.uint8)
    noise = []
    for p in (0.0, 0.01, 0.05, 0.06, 0.07, 0.08, 0.1, 0.11, 0.13, 0.15):
        tp, fp = roc.tp_fp(learn(roc.flip_noise(datab, p, seed + 17), ar, 4, None, 10000, seed), Tb)
        noise.append(dict(p=p, tp=tp, fp=fp))
    return {"roc_n20_ternary_m1000": roc_pts, "noise_n20_binary_m1000_10000_iters": noise,
            "note": "one chain per point; edges are directed m -> i; seeded synthetic data"}


def _ess_run(bn, torch, table, chains, seed, pre_steps, steps, stream, net=None, train_steps=0, thin=1):
    """ESS of the edge indicators over `steps` steps (every `thin`-th state recorded)
    after `pre_steps` uniform steps (and, for the learned sampler, `train_steps` of
    training on the history)."""
    ch = bn.chains_create(table, chains, seed, burn_in=pre_steps + train_steps, record_every=thin,
                          record_cap=(steps + thin - 1) // thin)
    bn.chains_step(ch, pre_steps, stream=stream.cuda_stream)
    t_train = 0.0
    if net is not None:
        bn.chains_set_proposal(ch, net, bn.PROPOSAL_TRAIN)
        t_train = _timed(bn, torch, ch, train_steps, stream) / 1000.0
        bn.chains_set_proposal(ch, net, bn.PROPOSAL_LEARNED, eps_mix=0.1)
    elif train_steps:
        bn.chains_step(ch, train_steps, stream=stream.cuda_stream)
    a0 = bn.chains_read(ch, "accepts").copy()
    sec = _timed(bn, torch, ch, steps, stream) / 1000.0
    acc = float((bn.chains_read(ch, "accepts") - a0).mean() / steps)
    f = bn.chains_read(ch, "edge_counts").sum(0) / (chains * steps)
    ess = bn.chains_read(ch, "ess")
    unc = (f >= 0.05) & (f <= 0.95) & ~np.isnan(ess)
    med = float(np.median(ess[unc])) if unc.any() else None
    mn = float(ess[unc].min()) if unc.any() else None
    ch.free()
    return dict(median_ess=med, min_ess=mn, uncertain_edges=int(unc.sum()), seconds=sec,
                ess_per_s=(med / sec) if med else None, acceptance=acc, steps=steps, chains=chains,
                train_seconds=t_train), f


def _batch_learned(bn, torch, synth, nets, tabs, seed, args):
    """The uneven batch with the learned proposal switched on for the largest network of
    each size class (n in 10-19, 20-29, 30-39, 40-49, 50-60), each trained first on its
    own chains' history, the others on the uniform swap in the shared fused launch; the
    same batch all-uniform beside it.  ESS of the edge indicators (every 10th state) per
    network; ESS/s = ESS over the whole batch's sampling time."""
    ns = [d_.shape[1] for d_, *_ in nets]
    pick = {}
    for i, nn in enumerate(ns):
        cls = min((nn - 10) // 10, 4)
        if cls not in pick or nn > ns[pick[cls]]:
            pick[cls] = i
    chains, steps, thin, train = 32, args.batch_ess_steps, 10, args.batch_train
    out = {"networks_learned": sorted(pick.values()), "n_learned": [ns[i] for i in sorted(pick.values())],
           "chains_per_network": chains, "steps": steps}
    for label in ("uniform", "learned"):
        bat = bn.batch_create(tabs, chains, seed + 6, burn_in=train, record_every=thin,
                              record_cap=(train + steps) // thin + 1)
        nets_keep = []
        if label == "learned":
            for i in pick.values():
                w = synth.mlp_init_weights(ns[i], 32, 512, seed + i)
                net = bn.mlp_create(ns[i], w, hidden=512, d=32, batch_cap=chains, lr=2e-3)
                nets_keep.append(net)
                bn.chains_set_proposal(bat.chains(i), net, bn.PROPOSAL_TRAIN, eps_mix=0.1)
                bn.chains_step(bat.chains(i), train)
                bn.chains_set_proposal(bat.chains(i), net, bn.PROPOSAL_LEARNED, eps_mix=0.1)
            others = [i for i in range(len(tabs)) if i not in pick.values()]
            for i in others:                              # the same step count as the learned ones
                bn.chains_step(bat.chains(i), train)
        else:
            bat.step(train)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        bat.step(steps)
        e1.record()
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1000.0
        per = []
        for i in sorted(pick.values()):
            f = bn.chains_read(bat.chains(i), "edge_counts").sum(0) / (chains * steps)
            ess = bn.chains_read(bat.chains(i), "ess")
            unc = (f >= 0.05) & (f <= 0.95) & ~np.isnan(ess)
            per.append(float(np.median(ess[unc])) if unc.any() else None)
        out[label] = {"seconds": sec, "order_evals_per_s": len(tabs) * chains * steps / sec,
                      "median_ess_of_learned_networks": per,
                      "ess_per_s": [e / sec if e else None for e in per]}
        bat.free()
        for net in nets_keep:
            net.free()
    out["note"] = ("learned networks step through their own three-kernel path after the shared fused launch "
                   "of the uniform networks (bn_batch_step); the all-uniform batch is the same networks, "
                   "chains and seeds")
    return out


def _oracle_configs(synth, nt, configs):
    """The oracle on all host cores at the other workloads: order evaluations/s on seeded
    random orders (n = 20 and n = 40 tables it builds itself), table entries/s of its
    build at n = 20, and the ESS/s its sampler would reach at n = 20: its trajectories are
    the library's step for step (tested), so its ESS per step is the library's and its
    ESS/s = that ESS x its steps/s."""
    import oracle
    out = {}
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    t0 = time.perf_counter()
    tab20 = oracle.build_table(data, arity, k, R=R, threads=nt)
    el = time.perf_counter() - t0
    out["n20_table_entries_per_s"] = tab20.size / el
    for name, tab, B in (("n20", tab20, 1000), ("n40", None, 10 * nt)):
        if tab is None:
            rng = np.random.Generator(np.random.PCG64(0xB4E50002))
            tab = rng.standard_normal((40, oracle.num_sets(39, 4))) * 10.0 - 500.0     # stand-in values
        orders = synth.random_orders(tab.shape[0], B, 7)
        t0 = time.perf_counter()
        oracle.order_scores(tab, 4, orders, threads=nt)
        el = time.perf_counter() - t0
        out[f"{name}_order_evals_per_s"] = B / el
    c20 = (configs or {}).get("n20_64chains") or {}
    if c20.get("ess_median"):
        per_step = c20["ess_median"] / 20000.0
        out["n20_ess_per_s"] = per_step * out["n20_order_evals_per_s"] / 64.0
    out["cores"] = nt
    out["note"] = ("n20: the oracle's own table (prior included); n40: a stand-in table of the shape (timing does "
                   "not depend on the values); 1,000 and 10 x cores orders")
    return out


def _config_n20(bn, torch, synth, seed):
    """20 ternary nodes, m = 1000, k = 4, with the pairwise prior (10 % of the true edges at
    +1, 10 % of the non-edges at -1); 64 chains x 20,000 iterations through the one-shot
    call, edge-posterior ESS from every 10th state."""
    data, arity, k, R, _ = synth.workload("n20_k4_m1000")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t = bn.build_scores(data, arity, k, R=R)
    bn.table_set_scan(t, bn.SCAN_PRUNED)
    torch.cuda.synchronize()
    prep = time.perf_counter() - t0
    chains, iters = 64, 20000
    bn.mcmc_run(t, chains, 2000, seed=seed + 20, burn_in=200)          # warm-up
    out = bn.mcmc_run(t, chains, iters, seed=seed + 21, burn_in=iters // 10, thin=10)
    st = out["stats"]
    t.free()
    return {"workload": "n20_k4_m1000 with the +-1 pairwise prior, 64 chains x 20,000 iterations",
            "order_evals_per_s": chains * iters / (st["sample_ms"] / 1000.0), "sample_ms": st["sample_ms"],
            "acceptance": st["acceptance"], "ess_median": st["ess_median"], "ess_min": st["ess_min"],
            "uncertain_edges": st["uncertain_edges"],
            "ess_per_s": st["ess_median"] / (st["sample_ms"] / 1000.0) if st["ess_median"] == st["ess_median"]
            else None, "table_and_prune_s": prep, "best_score": out["best_score"]}


def _config_n40(bn, torch, synth, seed, stream, flush, test_rate, hbm_peak):
    """40 ternary nodes, m = 2000, k = 4 (3.69 M entries): 512 chains stepped by the
    full-table scan, each step's three kernels replayed from a CUDA graph, on the tiling
    the autotuner picks for 512 items per node; the same chains on the pruned table's
    fused sampler beside it."""
    data, arity, k, R, _ = synth.workload("n40_k4_m2000")
    t = bn.build_scores(data, arity, k, R=R)
    S = bn.table_info(t)["sets_per_node"]
    n = data.shape[1]
    chains = 512
    sub, nchunk, tuned_us = bn.table_autotune(t, chains)
    with torch.cuda.stream(stream):
        ch = bn.chains_create(t, chains, seed + 40)
        bn.chains_step(ch, 5, stream=stream.cuda_stream)
        steps = 100
        ms = _timed(bn, torch, ch, steps, stream, pieces=steps, flush=flush)
        i0 = int(bn.chains_read(ch, "items")[0])
        scan_ms, scan_l = bn.chains_step_profiled(ch, 50, stream=stream.cuda_stream)
        items = int(bn.chains_read(ch, "items")[0]) - i0
        ch.free()
        tests = items * S / max(scan_l, 1)
        avg = scan_ms / max(scan_l, 1)
        bn.table_set_scan(t, bn.SCAN_PRUNED)
        fch = bn.chains_create(t, chains, seed + 41)
        bn.chains_step(fch, 1000, stream=stream.cuda_stream)
        fms = _timed(bn, torch, fch, 4000, stream, pieces=4, flush=flush)
        fch.free()
    t.free()
    return {"workload": "n40_k4_m2000, 512 chains", "full_table": {
                "order_evals_per_s": chains * steps / (ms / 1000.0), "ms_per_step": ms / steps,
                "tiling": {"stage_entries": sub, "blocks_per_node": nchunk, "tuned_us_per_launch": tuned_us},
                "scan_avg_ms": avg, "tests_per_s": tests / (avg / 1000.0),
                "test_frac": tests / (avg / 1000.0) / test_rate,
                "hbm_frac_algorithmic": (4 * n * S + 8 * S) / (avg / 1000.0) / 1e9 / hbm_peak,
                "note": "a step: predecessor lists + the scan + the MH update, replayed from a CUDA graph"},
            "pruned_fused": {"order_evals_per_s": chains * 4000 / (fms / 1000.0), "us_per_iteration": 1000.0 * fms / 4000}}


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import paper_1210_5128_gb300 as bn
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count

    stream = torch.cuda.Stream(device=dev)
    data, arity, k, R, _ = synth.workload(WORKLOAD)
    n = data.shape[1]

    # table build (preprocessing of Sec. III.A), timed on its own: the whole call by the
    # host clock, its counting-and-scoring kernel by CUDA events (a second build)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    table = bn.build_scores(data, arity, k, R=R)
    build_s = time.perf_counter() - t0
    t2, build_kernel_ms = bn.build_scores_profiled(data, arity, k, R=R)
    t2.free()
    S = bn.table_info(table)["sets_per_node"]
    seed = 0xC0FFEE + 7919 * rank

    # ---- bn_score_orders on a few orders: the full-table scan at memory speed -------------
    #      (the paper scores one order per MH iteration); device time of the scan kernel by
    #      CUDA events around its launch, L2 flushed before every call
    flush = (torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev),
             torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev))
    hbm_bytes = 4 * n * S + 8 * S            # sorted positions of every entry + the mask table once
    sliced_bytes = 4 * n * S                 # the parent-node bytes of every entry, in score order
    test_rate = bn.measure_test_rate()       # measured peak of the scan's consistency test
    # entries above (and including) each node's empty set in score order: all the sorted
    # mode can read
    tab_host = bn.table_scores(table)
    cut_entries = int(sum(int((tab_host[i] > tab_host[i, 0]).sum()) + 1 for i in range(n)))
    del tab_host

    def score_sweep(mode, batches):
        bn.table_set_scan(table, mode)
        out = []
        for B in batches:
            orders = torch.from_numpy(synth.random_orders(n, B, 100 + B)).to(dev)
            for _ in range(3):
                bn.score_orders_profiled(table, orders)
            times = []
            for _ in range(10 if B <= 64 else 5):
                _flush_l2(torch, flush, torch.cuda.current_stream())
                torch.cuda.synchronize()
                times.append(1000.0 * bn.score_orders_profiled(table, orders)[2])
            us = float(np.median(times))
            out.append({"orders": B, "scan_us": us, "scan_us_mean": float(np.mean(times)), "calls": len(times),
                        "order_evals_per_s": B / (us / 1e6)})
        bn.table_set_scan(table, bn.SCAN_FULL)
        return out

    hbm_leg = score_sweep(bn.SCAN_FULL, SCORE_B)
    for x in hbm_leg:
        B, us = x["orders"], x["scan_us"]
        tests = float(n) * S * B                 # (entry, order) consistency tests of one pass
        x.update({"kernel": "k_scan_nodes" if n * ((B + 7) // 8) <= 1024 else "k_scan",
                  "achieved_gbs": hbm_bytes / (us / 1e6) / 1e9, "frac": hbm_bytes / (us / 1e6) / 1e9 / hbm_peak,
                  "tests_per_s": tests / (us / 1e6), "test_frac": tests / (us / 1e6) / test_rate})
    sliced_leg = score_sweep(bn.SCAN_SLICED, SLICED_B)
    for x in sliced_leg:
        us = x["scan_us"]
        x.update({"kernel": "k_scan_sliced", "achieved_gbs": sliced_bytes / (us / 1e6) / 1e9,
                  "frac": sliced_bytes / (us / 1e6) / 1e9 / hbm_peak,
                  "tests_per_s": float(n) * S * x["orders"] / (us / 1e6)})
    sorted_leg = score_sweep(bn.SCAN_SORTED, SLICED_B)
    for x in sorted_leg:
        x.update({"kernel": "k_scan_sliced (early exit)", "entries_at_most": cut_entries})
    roof_b = ROOF_SLICED_B
    roof_sl = next(x for x in sliced_leg if x["orders"] == roof_b)

    # ---- the sum-based order score of the prior scorer (Sec. III.B) on the same table:
    #      one order, whole-call device time, L2 flushed before every call ------------------
    o1 = torch.from_numpy(synth.random_orders(n, 1, 101)).to(dev)
    bn.score_orders_sum(table, o1)
    sum_times = []
    for _ in range(5):
        _flush_l2(torch, flush, torch.cuda.current_stream())
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        bn.score_orders_sum(table, o1)
        e1.record()
        torch.cuda.synchronize()
        sum_times.append(1000.0 * e0.elapsed_time(e1))
    sum_score = {"orders": 1, "call_us": float(np.median(sum_times)),
                 "max_score_scan_us": hbm_leg[0]["scan_us"],
                 "note": "bn_score_orders_sum: FP64 log10-sum-exp10 over the consistent parent sets of "
                         "every node (one exp10 per consistent set), against the max-based scan of the "
                         "same order (roofline_hbm)"}

    with torch.cuda.stream(stream):
        # ---- full-table scan sampler ----------------------------------------------------
        full = bn.chains_create(table, args.chains, seed=seed)
        bn.chains_step(full, args.warmup, stream=stream.cuda_stream)
        i0 = int(bn.chains_read(full, "items")[0])
        ms_full = _timed(bn, torch, full, args.steps, stream, pieces=args.steps, flush=flush)
        items_full = int(bn.chains_read(full, "items")[0]) - i0
        prof_steps = max(20, min(args.steps, 100))
        i1 = int(bn.chains_read(full, "items")[0])
        scan_ms_full, scan_l_full = bn.chains_step_profiled(full, prof_steps, stream=stream.cuda_stream)
        items_prof = int(bn.chains_read(full, "items")[0]) - i1
        full.free()

        # ---- the same full scan with every parent set unranked on the fly (no table) --------
        bn.table_set_scan(table, bn.SCAN_UNRANK)
        unr = bn.chains_create(table, args.chains, seed=seed)
        bn.chains_step(unr, args.warmup, stream=stream.cuda_stream)
        unr_steps = max(3, min(args.steps, 50))
        ms_unr = _timed(bn, torch, unr, unr_steps, stream, pieces=unr_steps, flush=flush)
        unr.free()
        # ---- the same steps on the bit-sliced scans: every entry, and stopping early -------
        sl_samp = {}
        for name, mode in (("sliced", bn.SCAN_SLICED), ("sorted", bn.SCAN_SORTED)):
            bn.table_set_scan(table, mode)
            chs = bn.chains_create(table, args.chains, seed=seed)
            bn.chains_step(chs, args.warmup, stream=stream.cuda_stream)
            ms_sl = _timed(bn, torch, chs, args.steps, stream, pieces=args.steps, flush=flush)
            sl_ms, sl_l = bn.chains_step_profiled(chs, prof_steps, stream=stream.cuda_stream)
            chs.free()
            sl_samp[name] = {"value": world * args.chains * args.steps / (ms_sl / 1000.0),
                             "ms_per_step": ms_sl / args.steps, "scan_avg_ms": sl_ms / max(sl_l, 1)}
        bn.table_set_scan(table, bn.SCAN_FULL)

        # ---- pruned scan sampler (headline) ----------------------------------------------
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bn.table_set_scan(table, bn.SCAN_PRUNED)
        prune_s = time.perf_counter() - t0
        survivors = bn.table_pruned(table)
        ips = args.iters_per_step
        chains = bn.chains_create(table, args.chains, seed=seed)
        bn.chains_step(chains, args.warmup * ips, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        barrier()
        clk = ClockSampler(local)
        clk.start()
        l0 = bn.kernel_launches()
        it0 = int(bn.chains_read(chains, "items")[0])
        ms = _timed(bn, torch, chains, args.steps * ips, stream, pieces=args.steps, flush=flush)
        launches = bn.kernel_launches() - l0
        items_head = int(bn.chains_read(chains, "items")[0]) - it0
        barrier()
        clocks = clk.stop()
        # the fused sampler kernel, launch by launch (up to 1024 iterations per launch)
        fused_ms, fused_l = bn.chains_step_profiled(chains, max(ips, 256) * 4, stream=stream.cuda_stream)
        chains.free()
        # the same kernel with one chain: its block alone on the GPU, nothing competing for
        # its SM -- the dependent-latency floor of this code's MH step
        solo = bn.chains_create(table, 1, seed=seed + 99)
        bn.chains_step(solo, 2 * max(ips, 256), stream=stream.cuda_stream)
        solo_ms, solo_l = bn.chains_step_profiled(solo, max(ips, 256) * 4, stream=stream.cuda_stream)
        solo.free()

    # ---- bn_score_orders on the pruned table (only entries no subset matches or beats) -----
    pruned_scoring = []
    for B in (1, 64, 1024, 8192):
        orders = torch.from_numpy(synth.random_orders(n, B, 300 + B)).to(dev)
        for _ in range(3):
            bn.score_orders_profiled(table, orders)
        times = []
        for _ in range(10):
            _flush_l2(torch, flush, torch.cuda.current_stream())
            torch.cuda.synchronize()
            times.append(1000.0 * bn.score_orders_profiled(table, orders)[2])
        us = float(np.median(times))
        pruned_scoring.append({"orders": B, "scan_us": us, "order_evals_per_s": B / (us / 1e6)})

    t_max = ms
    if world > 1:
        tt = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    value = world * args.chains * args.steps * ips / (t_max / 1000.0)

    # ---- edge-posterior ESS/s: plain vs learned proposal (same table, same chains) --------
    ess = None
    if not args.no_ess and rank == 0:
        with torch.cuda.stream(stream):
            pre = 300
            plain, f_plain = _ess_run(bn, torch, table, args.chains, seed + 1, pre, args.ess_steps, stream,
                                      train_steps=args.train_steps, thin=args.ess_thin)
            d, H = 32, 512
            net = bn.mlp_create(n, synth.mlp_init_weights(n, d, H, seed), hidden=H, d=d, batch_cap=args.chains,
                                lr=2e-3)
            learned, f_learned = _ess_run(bn, torch, table, args.chains, seed + 2, pre, args.ess_steps, stream,
                                          net=net, train_steps=args.train_steps, thin=args.ess_thin)
            # long plain run (8x) as the reference for the learned sampler's edge frequencies
            long_ch = bn.chains_create(table, args.chains, seed + 3, burn_in=pre)
            bn.chains_step(long_ch, pre + 8 * args.ess_steps, stream=stream.cuda_stream)
            f_long = bn.chains_read(long_ch, "edge_counts").sum(0) / (args.chains * 8 * args.ess_steps)
            long_ch.free()
        ess = {"plain": plain, "learned": learned,
               "max_abs_edge_freq_diff_learned_vs_long_plain": float(np.abs(f_learned - f_long).max()),
               "max_abs_edge_freq_diff_plain_vs_long_plain": float(np.abs(f_plain - f_long).max()),
               "long_plain_steps": 8 * args.ess_steps,
               "learned_over_plain_ess_per_s": (learned["ess_per_s"] / plain["ess_per_s"])
               if learned["ess_per_s"] and plain["ess_per_s"] else None}

    # ---- uneven batch: 96 networks (n 10..60, arity 2..4, m 200..5000, k 3..4), 32 chains
    #      each, every network's chains in one fused launch --------------------------------
    batch = None
    if not args.no_batch and rank == 0:
        nets = synth.uneven_batch(96, 0xB4E50000 + 4)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tabs = [bn.build_scores(d_, a_, k_, R=r_) for d_, a_, k_, r_, _ in nets]
        torch.cuda.synchronize()
        b_build = time.perf_counter() - t0
        b_entries = sum(bn.table_info(tb)["n"] * bn.table_info(tb)["sets_per_node"] for tb in tabs)
        for tb in tabs:
            bn.table_set_scan(tb, bn.SCAN_PRUNED)
        bat = bn.batch_create(tabs, 32, seed + 5)
        bat.step(256)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        bat.step(args.batch_iters)
        e1.record()
        torch.cuda.synchronize()
        b_ms = e0.elapsed_time(e1)
        b_chains = 96 * 32
        batch = {"networks": 96, "chains_per_network": 32, "iterations": args.batch_iters,
                 "order_evals_per_s": b_chains * args.batch_iters / (b_ms / 1000.0), "ms": b_ms,
                 "n_range": [min(d_.shape[1] for d_, *_ in nets), max(d_.shape[1] for d_, *_ in nets)],
                 "table_entries": int(b_entries), "table_build_s": b_build,
                 "table_entries_per_s": b_entries / b_build,
                 "note": "uniform-swap chains of every network in one fused launch per 1024 steps "
                         "(bn_batch_step); the learned proposal runs per network (bn_chains_set_proposal)"}
        bat.free()
        batch["learned_per_size_class"] = _batch_learned(bn, torch, synth, nets, tabs, seed, args)
        for tb in tabs:
            tb.free()
        del tabs

    # ---- the other configurations of the metric's workload family ---------------------------
    configs = None
    if rank == 0 and not args.no_configs:
        configs = {"n20_64chains": _config_n20(bn, torch, synth, seed),
                   "n40_512chains": _config_n40(bn, torch, synth, seed, stream, flush, test_rate, hbm_peak)}

    # ---- accuracy study (Sec. VI): ROC points with the prior schedule, noise tolerance ----
    accuracy = _accuracy(bn, synth, 29) if (rank == 0 and not args.no_accuracy) else None

    # ---- end to end through the public C ABI with host buffers ----------------------------
    e2e_steps = max(50, args.steps) * args.iters_per_step
    e2e_calls = 2
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in range(e2e_calls):
        tb = bn.build_scores(data, arity, k, R=R)
        bn.table_set_scan(tb, bn.SCAN_PRUNED)
        out = bn.mcmc_run(tb, args.chains, e2e_steps, seed=17 + c, burn_in=e2e_steps // 10)
        tb.free()
    e2e_s = (time.perf_counter() - t0) / e2e_calls
    e2e_value = world * args.chains * e2e_steps / e2e_s
    h2d = data.nbytes + arity.nbytes + (R.nbytes if R is not None else 0)
    d2h = out["best_order"].nbytes + out["best_dag"].nbytes + 8 + out["edge_freq"].nbytes

    if rank == 0:
        clock_mhz = (clocks or {}).get("sm_mhz") or 2070.0
        avg_fused = fused_ms / max(fused_l, 1)
        iters_fused = max(ips, 256) * 4 / max(fused_l, 1)              # MH iterations per profiled launch
        inst = FUSED_INST_PER_CHAIN_STEP * args.chains * iters_fused   # warp instructions per launch
        issue_peak = n_sm * ISSUE_PER_SM * clock_mhz * 1e6
        roof_head = {"kernel": "k_chain_spec<1> (the timed step: pruned table, four warps per chain evaluating "
                               "consecutive MH steps at once, up to 1,024 MH iterations per launch)",
                     "bound": "alu", "unit": "warp instructions/s",
                     "achieved": inst / (avg_fused / 1000.0), "peak": issue_peak,
                     "frac": inst / (avg_fused / 1000.0) / issue_peak, "traffic": FUSED_TRAFFIC_BYTES,
                     "peak_source": f"derived: {n_sm} SMs x {ISSUE_PER_SM} schedulers x 1 warp instruction per "
                                    f"clock x {clock_mhz:.0f} MHz (SM clock sampled in the timed region)",
                     "per_launch": {"avg_ms": avg_fused, "launches": fused_l, "iterations": iters_fused,
                                    "warp_instructions": inst,
                                    "warp_instructions_per_chain_iteration": FUSED_INST_PER_CHAIN_STEP,
                                    "us_per_iteration": 1000.0 * avg_fused / iters_fused},
                     "latency_floor": {"us_per_iteration_one_chain": 1000.0 * solo_ms / (max(ips, 256) * 4),
                                       "frac": (solo_ms / (max(ips, 256) * 4)) / (avg_fused / iters_fused),
                                       "note": "the same kernel and table with a single chain (one block of four "
                                               "warps alone on the GPU): the dependent-latency floor of this MH "
                                               "step's code; frac = floor / the 256-chain time per iteration"},
                     "note": "latency-bound: 256 chains are 1,024 warps on 152 SMs; a round of a chain's four "
                             "warps is a chain of dependent shared-memory loads, shuffles and votes, and ends at "
                             "the slowest warp's evaluation and the accepted step's update (ncu: barrier and "
                             "fixed-latency stalls lead), so issue slots stay idle; the instruction count per "
                             "committed chain-iteration is ncu's smsp__inst_executed.sum for this kernel at this "
                             "workload, speculative evaluations included; DRAM traffic is the survivors' and "
                             "chains' state only (the table stays in shared memory)"}
        avg_full = scan_ms_full / max(scan_l_full, 1)
        tests = items_prof * S / max(scan_l_full, 1)                 # (entry, item) tests per launch
        roof_scan = {"kernel": "k_scan (full table, autotuned tiling, one launch per sampler step of all chains)",
                     "bound": "alu", "unit": "tests/s", "achieved": tests / (avg_full / 1000.0),
                     "peak": test_rate, "frac": tests / (avg_full / 1000.0) / test_rate,
                     "traffic": SCAN_TRAFFIC_BYTES,
                     "peak_source": "measured in this run: bn_measure_test_rate (the scan's own inner loop over "
                                    "1,024 entries resident in shared memory, 8 x 256 threads per SM, CUDA events)",
                     "per_launch": {"tests": tests, "avg_ms": avg_full, "launches": scan_l_full,
                                    "hbm_bytes_algorithmic": 4 * n * S + 8 * S,
                                    "hbm_frac_of_measured": (4 * n * S + 8 * S) / (avg_full / 1000.0) / 1e9 / hbm_peak},
                     "share_of_step": avg_full / (ms_full / args.steps),
                     "note": "the paper's scan (a6) over the full table for a step of all chains' orders "
                             "(full_scan): the table is read once per 256 orders, so the consistency tests, "
                             "not HBM, bound it; traffic = ncu dram bytes read + written per launch"}
        cpu = cpu1 = None
        if world == 1 and not args.no_cpu_baseline:
            nt = os.cpu_count() or 1
            rate, done, el, used = oracle_sample(args.cpu_seconds, threads=nt)
            cpu = {"value": rate, "unit": UNIT, "cores": used, "kind": "oracle",
                   "sample": f"{done} order evaluations ({el:.1f} s) of the oracle's MH sampler at n=60, k=4 "
                             f"(full order score per iteration), {used} chains at a time in {used} host threads "
                             f"of the {nt} cores, on a seeded stand-in table of the workload's shape"}
            rate1, done1, el1, _ = oracle_sample(args.cpu_seconds / 2, threads=1)
            cpu1 = {"value": rate1, "unit": UNIT, "cores": 1, "kind": "oracle",
                    "sample": f"{done1} order evaluations ({el1:.1f} s), one thread"}
            cpu["configs"] = _oracle_configs(synth, nt, configs)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": run_config(args),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "note": f"per call: bn_build_scores from host data + pruning + bn_mcmc_run of {e2e_steps} "
                            f"steps x {args.chains} chains + results to host"},
            "gpu_launches": int(launches),
            "work_per_iteration": {"order_evals": args.chains,
                                   "nodes_rescored": items_head / (args.steps * ips),
                                   "survivors_per_node_mean": float(survivors.mean()),
                                   "note": "every iteration scores a full order of each chain; only the nodes "
                                           "between the swapped positions are re-scored (the others keep their "
                                           "parent sets), each over its surviving entries in score order"},
            "roofline": roof_head,
            "roofline_scan": roof_scan,
            "roofline_build": {"kernel": "k_build<4,1,0> (counting + local score + prior of every entry, n=60)",
                               "bound": "alu", "unit": "warp instructions/s",
                               "achieved": BUILD_INST_PER_ENTRY * n * S / (build_kernel_ms / 1000.0),
                               "peak": issue_peak,
                               "frac": BUILD_INST_PER_ENTRY * n * S / (build_kernel_ms / 1000.0) / issue_peak,
                               "traffic": None, "kernel_ms": build_kernel_ms,
                               "row_visits_per_s": n * S * data.shape[0] / (build_kernel_ms / 1000.0),
                               "note": "issue-bound: warp instructions per entry = ncu smsp__inst_executed.sum of "
                                       "this kernel at this workload (649); peak as for roofline; DRAM carries only "
                                       "the 8 B written per entry"},
            "roofline_hbm": {"kernel": f"k_scan_sliced (bn_score_orders, BN_SCAN_SLICED: every entry of the full "
                                       f"table, {roof_b} orders)", "bound": "hbm",
                             "achieved": roof_sl["achieved_gbs"], "peak": hbm_peak, "unit": "GB/s",
                             "frac": roof_sl["frac"], "traffic": SLICED_TRAFFIC_BYTES, "peak_source": peak_src,
                             "bytes_algorithmic": sliced_bytes, "orders": roof_b,
                             "note": "batched scoring over the full table: every entry of every node streamed once "
                                     "for 32 orders; algorithmic bytes = 4 B (the parent-node bytes) per (node, "
                                     "entry); traffic = ncu dram bytes read + written for this launch shape; bound "
                                     "in practice by the per-entry tests of the slowest blocks (ncu: 0.5 of the "
                                     "issue slots busy, DRAM below peak)"},
            "roofline_hbm_one_order": {"kernel": "k_scan_nodes (bn_score_orders, BN_SCAN_FULL, one order)",
                                       "bound": "hbm", "achieved": hbm_leg[0]["achieved_gbs"], "peak": hbm_peak,
                                       "unit": "GB/s", "frac": hbm_leg[0]["frac"], "bytes_algorithmic": hbm_bytes,
                                       "traffic": NODES_TRAFFIC_BYTES},
            "score_orders": {"by_orders": hbm_leg, "sliced": sliced_leg, "sorted": sorted_leg,
                             "test_rate_peak": test_rate, "pruned_table": pruned_scoring,
                             "note": "bn_score_orders on B random orders of the full n=60 table: scan kernel time "
                                     "(CUDA events around its launch, L2 flushed before every call). by_orders: "
                                     "BN_SCAN_FULL (one 64-bit mask test per entry and order), HBM fraction on 4 B "
                                     "per (node, entry) + 8 B per entry, test fraction of the measured "
                                     "consistency-test peak; sliced: BN_SCAN_SLICED (entries in score order, 32 "
                                     "orders per AND of parent words; every entry read), HBM fraction on 4 B per "
                                     "(node, entry); sorted: BN_SCAN_SORTED (the same, nothing below the empty set "
                                     "read, stopping once every order has its entry; entries_at_most = the entries "
                                     "above the empty sets); pruned_table: the table keeping only the entries no "
                                     "subset matches or beats. All modes give identical results"},
            "pruned_step": {"kernel": "k_chain_spec (up to 1024 MH iterations per launch, four warps per chain)",
                            "avg_ms_per_launch": avg_fused, "launches": fused_l,
                            "us_per_iteration": 1000.0 * fused_ms / max(ips, 256) / 4,
                            "survivors_per_node_mean": float(survivors.mean()),
                            "survivors_per_node_max": int(survivors.max()),
                            "survivor_fraction": float(survivors.sum() / (n * S)), "prune_s": prune_s},
            "full_scan": {"value": world * args.chains * args.steps / (ms_full / 1000.0),
                          "ms_per_step": ms_full / args.steps, "items_per_step": items_full / args.steps,
                          "sliced": dict(sl_samp["sliced"], note="BN_SCAN_SLICED: the bit-sliced full pass"),
                          "sorted": dict(sl_samp["sorted"], note="BN_SCAN_SORTED: bit-sliced, stopping early"),
                          "unranked_sets": {"value": world * args.chains * unr_steps / (ms_unr / 1000.0),
                                            "ms_per_step": ms_unr / unr_steps, "steps": unr_steps,
                                            "note": "BN_SCAN_UNRANK: every parent set computed from its rank "
                                                    "in the scan instead of read from the parent-set table"}},
            "ess": ess,
            "sum_score": sum_score,
            "uneven_batch": batch,
            "accuracy": accuracy,
            "configs": configs,
            "cpu_baseline": cpu,
            "cpu_baseline_1core": cpu1,
            "clocks": clocks,
            "table_build_s": build_s,
            "table_entries_per_s": n * S / build_s,
            "table_row_visits_per_s": n * S * data.shape[0] / build_s,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
