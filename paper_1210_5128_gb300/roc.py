"""Accuracy of learned graphs (Sec. VI, the ROC study of Figs. 8-10).

Host-side bookkeeping around the sampler; no arithmetic of the method lives here.

- ``tp_fp(learned, true)``: true-positive rate = found true edges / true edges, false-positive
  rate = wrongly added edges / non-edges, over directed edges m -> i (i != m); adjacency
  matrices are [i][m] = 1 iff m -> i, as ``bn_mcmc_run`` returns them.  The skeleton
  variant ignores edge direction.
- ``prior_from_errors``: the paper's prior schedule for the second to fifth ROC points: the
  edges a prior-free run missed get R = r_missed (0.7 or 0.8) and the edges it added wrongly
  get R = r_added (0.2 or 0.1), each with probability ``prob`` (0.2 or 0.4); every other
  pair stays at R = 0.5 (no prior).
- ``flip_noise``: every value of a binary data set flips with probability p (the noise
  study of Fig. 10).
"""
from __future__ import annotations

import numpy as np

__all__ = ["tp_fp", "prior_from_errors", "flip_noise", "true_adjacency"]


def _offdiag(n):
    return ~np.eye(n, dtype=bool)


def tp_fp(learned, true, skeleton=False):
    """(TP rate, FP rate) of a learned adjacency against the true one."""
    L = np.asarray(learned, bool)
    T = np.asarray(true, bool)
    n = T.shape[0]
    off = _offdiag(n)
    if skeleton:
        L = L | L.T
        T = T | T.T
        off = np.triu(off)
    pos = T & off
    neg = ~T & off
    tp = (L & pos).sum() / max(pos.sum(), 1)
    fp = (L & neg).sum() / max(neg.sum(), 1)
    return float(tp), float(fp)


def true_adjacency(net):
    """[i][m] = 1 iff m is a parent of i in a network from ``synth.random_network``."""
    n = len(net.parents)
    A = np.zeros((n, n), np.uint8)
    for i, ps in enumerate(net.parents):
        for m in ps:
            A[i, m] = 1
    return A


def prior_from_errors(learned, true, r_missed, r_added, prob, seed):
    """Prior matrix R (n x n, [i][m] = prior on m -> i) built from a prior-free run's
    errors: missed true edges get r_missed, wrongly added edges r_added, each with
    probability ``prob`` (a seeded draw per edge); all else 0.5."""
    L = np.asarray(learned, bool)
    T = np.asarray(true, bool)
    n = T.shape[0]
    off = _offdiag(n)
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random((n, n))
    R = np.full((n, n), 0.5)
    R[T & ~L & off & (u < prob)] = r_missed
    R[~T & L & off & (u < prob)] = r_added
    return R


def flip_noise(data, p, seed):
    """Binary data with every value flipped with probability p."""
    d = np.asarray(data, np.uint8)
    rng = np.random.Generator(np.random.PCG64(seed))
    return (d ^ (rng.random(d.shape) < p).astype(np.uint8)).astype(np.uint8)
