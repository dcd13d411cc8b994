#!/usr/bin/env python
"""Throughput of the order-space MH sampler (Algorithm 1) on one GB300.

One step = one Metropolis-Hastings iteration of every chain: a swap proposal per chain,
the order score of Eq. (6) of every proposed order (an exact full-order score; only the
nodes between the swapped positions are re-scanned, the others keep their best sets),
the MH test, best-graph and edge-count updates -- three kernels replayed from a CUDA
graph.  Workload: 60 ternary nodes, in-degree <= 3, m = 1000 synthetic samples, k = 4
(489,406 parent sets per node, 29.36 M FP64 entries, 235 MB), 256 chains.

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
                                          "--format=csv,noheader,nounits", "-lms", "100"],
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


def oracle_sample(seconds):
    """The oracle's sampler (Algorithm 1: a full order score per iteration) at n = 60,
    k = 4, run in short single-chain batches until ``seconds`` have passed."""
    import oracle
    tab, k = _standin_table()
    done, c, t0 = 0, 0, time.perf_counter()
    while True:
        oracle.mcmc_run(tab, k, 1, 4, seed=1000 + c)
        done += 5                 # the initial order + 4 proposals
        c += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            return done / el, done, el


def run_reference(args):
    """Reference arm: the oracle as it stands on one host core.  One step = one order
    evaluation (Eq. 6 by the oracle's brute-force subset walk) of a random order of the
    n = 60, k = 4 workload."""
    import oracle
    import synth
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    tab, k = _standin_table()
    orders = synth.random_orders(60, args.steps + 2, 4242)
    for i in range(min(args.warmup, 2)):
        oracle.order_score(tab, k, orders[i])
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle.order_score(tab, k, orders[2 + i])
    tot = time.perf_counter() - t0
    value = args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(args.chains),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} order evaluations ({tot:.1f} s) by the oracle at n=60, k=4, "
                                   "one per step, on a seeded stand-in table of the workload's shape"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def config_dict(chains):
    return {"workload": f"{WORKLOAD}: 60 ternary nodes, random DAG in-degree<=3, m=1000 synthetic samples, "
                        f"k=4 (489,406 parent sets/node, 29.36M FP64 entries, 235 MB), {chains} chains, "
                        "uniform swap proposal",
            "chains": chains, "n": 60, "k": 4, "m": 1000,
            "l2": "inputs larger than L2 (235 MB table streamed per step)"}


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

    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    data, arity, k, R, _ = synth.workload(WORKLOAD)
    n = data.shape[1]

    # table build (preprocessing of Sec. III.A), timed on its own
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    table = bn.build_scores(data, arity, k, R=R)
    build_s = time.perf_counter() - t0
    info = bn.table_info(table)
    S = info["sets_per_node"]

    chains = bn.chains_create(table, args.chains, seed=0xC0FFEE + 7919 * rank, burn_in=0)
    with torch.cuda.stream(stream):
        bn.chains_step(chains, args.warmup, stream=sp)
        torch.cuda.synchronize()
        barrier()
        clk = ClockSampler(local)
        clk.start()
        l0 = bn.kernel_launches()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        bn.chains_step(chains, args.steps, stream=sp)
        e1.record(stream)
        torch.cuda.synchronize()
        launches = bn.kernel_launches() - l0
        barrier()
        clocks = clk.stop()
        ms = e0.elapsed_time(e1)
        # dominant kernel: the scan, timed launch by launch with events on this stream
        prof_steps = max(20, min(args.steps, 200))
        scan_ms, scan_launches = bn.chains_step_profiled(chains, prof_steps, stream=sp)
    t_max = ms
    if world > 1:
        tt = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    evals = world * args.chains * args.steps
    value = evals / (t_max / 1000.0)

    # end to end through the public C ABI with host buffers: table build from host data
    # + a run of the sampler + results copied back, every call
    e2e_steps = max(50, args.steps // 2)
    e2e_calls = 2
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in range(e2e_calls):
        tb = bn.build_scores(data, arity, k, R=R)
        out = bn.mcmc_run(tb, args.chains, e2e_steps, seed=17 + c, burn_in=e2e_steps // 10)
        tb.free()
    e2e_s = (time.perf_counter() - t0) / e2e_calls
    e2e_value = world * args.chains * e2e_steps / e2e_s
    h2d = data.nbytes + arity.nbytes + (R.nbytes if R is not None else 0)
    d2h = out["best_order"].nbytes + out["best_dag"].nbytes + 8 + out["edge_freq"].nbytes

    line = None
    if rank == 0:
        avg_scan = scan_ms / max(scan_launches, 1)
        alg_bytes = 8 * n * S
        achieved = alg_bytes / (avg_scan / 1000.0) / 1e9
        roof = {"kernel": "k_scan", "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None,
                "peak_source": f"{peak_src} hbm_gbs",
                "per_launch": {"algorithmic_bytes": alg_bytes, "avg_ms": avg_scan, "launches": scan_launches},
                "share_of_step": (scan_ms / scan_launches) / (ms / args.steps)}
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            rate, done, el = oracle_sample(args.cpu_seconds)
            cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{done} order evaluations ({el:.1f} s) of the oracle's MH sampler at n=60, k=4, "
                             "full order score per iteration, on a seeded stand-in table of the workload's shape"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args.chains),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "note": f"per call: bn_build_scores from host data + bn_mcmc_run of {e2e_steps} steps x "
                            f"{args.chains} chains + results to host"},
            "gpu_launches": int(launches),
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "table_build_s": build_s,
            "table_entries_per_s": n * S / build_s,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
