"""The multi-GPU path is replicas of independent chains merged once at the end.  Its host
logic runs here as two gloo ranks on CPU: each rank samples its own chains (the oracle's
sampler stands in for a GPU replica), the merge must equal the combination computed in
one process."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_results(rank):
    data, arity, k, R, _ = synth.workload("n6_k2_m100")
    tab = oracle.build_table(data, arity, k, R=R)
    return oracle.mcmc_run(tab, k, 3, 400, seed=1000 + rank, burn_in=50)


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    from paper_1210_5128_gb300.replicas import merge_replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r = _rank_results(rank)
    ec, bs, bo, br, src = merge_replicas(r["edge_counts"], r["best_score"], r["best_order"], r["best_rank"])
    np.savez(os.path.join(out_dir, f"r{rank}.npz"), ec=ec, bs=bs, bo=bo, br=br, src=src)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_merge(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = [_rank_results(r) for r in range(world)]
    ec = sum(r["edge_counts"].sum(0).astype(np.int64) for r in res)
    best = [(r["best_score"].max(), i) for i, r in enumerate(res)]
    bs, src = max(best, key=lambda x: (x[0], -x[1]))
    c = int(np.argmax(res[src]["best_score"]))
    for rank in range(world):
        z = np.load(tmp_path / f"r{rank}.npz")
        assert np.array_equal(z["ec"], ec)            # both ranks hold the merged counts
        assert float(z["bs"]) == bs and int(z["src"]) == src
        assert np.array_equal(z["bo"], res[src]["best_order"][c])
        assert np.array_equal(z["br"], res[src]["best_rank"][c])
