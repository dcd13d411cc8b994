"""Merging independent sampler replicas across ranks.

The sampler's chains are independent, so several GPUs run replicas -- each its own copy
of the table and its own chains -- with no exchange during sampling.  At the end the
per-rank results are merged once on the host side of torch.distributed:

* edge counts are summed (so edge frequencies are over all ranks' chains and steps);
* the best graph is the one with the highest best score, ties to the lowest rank and then
  the lowest chain, matching the single-GPU rule (lowest chain id on ties).

Works with any process-group backend (gloo on CPU tensors, nccl on CUDA tensors).
"""
from __future__ import annotations

import numpy as np


def merge_replicas(edge_counts, best_scores, best_orders, best_ranks, group=None):
    """edge_counts (C, n, n) integer counts of this rank's chains; best_scores (C,),
    best_orders (C, n), best_ranks (C, n) of this rank.  Returns (edge_counts_total (n, n)
    int64 over all ranks, best_score, best_order (n,), best_rank (n,), best_rank_of)."""
    import torch
    import torch.distributed as dist

    ec = torch.as_tensor(np.asarray(edge_counts, np.int64).sum(axis=0))
    dist.all_reduce(ec, op=dist.ReduceOp.SUM, group=group)
    bs = np.asarray(best_scores, np.float64)
    c = int(np.argmax(bs))                         # lowest chain id among equal maxima
    mine = torch.tensor([bs[c]], dtype=torch.float64)
    world = dist.get_world_size(group)
    scores = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(scores, mine, group=group)
    vals = [float(s.item()) for s in scores]
    src = int(np.argmax(vals))                     # lowest rank among equal maxima
    payload = torch.as_tensor(np.concatenate([np.asarray(best_orders, np.int64)[c],
                                              np.asarray(best_ranks, np.int64)[c]]))
    dist.broadcast(payload, src=dist.get_global_rank(group, src) if group is not None else src, group=group)
    n = np.asarray(best_orders).shape[1]
    p = payload.numpy()
    return ec.numpy(), vals[src], p[:n].astype(np.uint8), p[n:].astype(np.uint32), src
