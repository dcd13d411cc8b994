"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no arithmetic of the learning method (no counting, no scores, no
order scoring, no sampler).  It only draws the inputs those consume:

* a random DAG with a bounded in-degree over ``n`` discrete variables, CPT rows from a
  Dirichlet(1) distribution, and ``m`` forward samples (the paper assumes complete,
  multinomial, observational data, Sec. II);
* the pairwise prior interface matrix ``R`` of Sec. IV (``R[i, m]`` is the belief in an
  edge ``v_m -> v_i``; 0.5 = no bias), drawn as a "confidence" ``c`` in {-1, 0, +1}
  mapped to ``R = (1 + c) / 2``;
* random node orders (position -> node).

All draws use numpy's PCG64 generator with an explicit seed, so every caller that asks
for the same workload receives byte-identical arrays.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Network",
    "random_network",
    "forward_sample",
    "prior_matrix",
    "random_orders",
    "workload",
    "WORKLOADS",
]


@dataclasses.dataclass
class Network:
    n: int
    arity: np.ndarray            # (n,) uint8, states per variable (2..4)
    parents: list                # parents[i] = sorted list of parent node ids
    cpt: list                    # cpt[i] = (q_i, r_i) float64 rows, sum to 1
    topo: np.ndarray             # (n,) a topological order of the true DAG

    def adjacency(self) -> np.ndarray:
        """(n, n) uint8, ``adj[i, m] = 1`` iff the true DAG has the edge m -> i."""
        a = np.zeros((self.n, self.n), np.uint8)
        for i, ps in enumerate(self.parents):
            for p in ps:
                a[i, p] = 1
        return a


def random_network(n: int, max_indeg: int, arity, seed: int) -> Network:
    """Random DAG: a uniform random topological order; the node at position p draws an
    in-degree d ~ U{0..min(max_indeg, p)} and d distinct parents uniformly among the
    nodes before it.  CPT rows ~ Dirichlet(1).  ``arity`` is an int (all nodes) or an
    array of per-node arities."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if np.isscalar(arity):
        ar = np.full(n, int(arity), np.uint8)
    else:
        ar = np.asarray(arity, np.uint8).copy()
        assert ar.shape == (n,)
    topo = rng.permutation(n)
    parents = [[] for _ in range(n)]
    for p in range(n):
        node = int(topo[p])
        d = int(rng.integers(0, min(max_indeg, p) + 1))
        if d:
            ps = rng.choice(topo[:p], size=d, replace=False)
            parents[node] = sorted(int(x) for x in ps)
    cpt = []
    for i in range(n):
        q = int(np.prod([int(ar[p]) for p in parents[i]], dtype=np.int64)) if parents[i] else 1
        cpt.append(rng.dirichlet(np.ones(int(ar[i])), size=q))
    return Network(n=n, arity=ar, parents=parents, cpt=cpt, topo=topo)


def forward_sample(net: Network, m: int, seed: int) -> np.ndarray:
    """``m`` ancestral samples of ``net`` as an (m, n) uint8 row-major array.  A row's
    parent configuration index is mixed radix with the first (lowest-id) parent least
    significant; the child state is drawn by inverse CDF from the CPT row."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.zeros((m, net.n), np.uint8)
    for node in net.topo:
        node = int(node)
        cfg = np.zeros(m, np.int64)
        stride = 1
        for p in net.parents[node]:
            cfg += x[:, p].astype(np.int64) * stride
            stride *= int(net.arity[p])
        cdf = np.cumsum(net.cpt[node], axis=1)
        u = rng.random(m)
        v = (u[:, None] >= cdf[cfg]).sum(axis=1)
        x[:, node] = np.minimum(v, int(net.arity[node]) - 1).astype(np.uint8)
    return x


def prior_matrix(net: Network, frac_true: float, frac_false: float, seed: int) -> np.ndarray:
    """Pairwise prior interface matrix (Sec. IV): a fraction ``frac_true`` of the true
    edges get confidence +1 (R = 1), a fraction ``frac_false`` of the non-edges get -1
    (R = 0), the rest 0 (R = 0.5).  Row = child, column = parent; diagonal 0.5."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = net.n
    adj = net.adjacency()
    conf = np.zeros((n, n), np.float64)
    true_e = [(i, j) for i in range(n) for j in range(n) if i != j and adj[i, j]]
    false_e = [(i, j) for i in range(n) for j in range(n) if i != j and not adj[i, j]]
    for lst, c, fr in ((true_e, 1.0, frac_true), (false_e, -1.0, frac_false)):
        k = int(round(fr * len(lst)))
        if k:
            pick = rng.choice(len(lst), size=k, replace=False)
            for t in pick:
                i, j = lst[int(t)]
                conf[i, j] = c
    return (1.0 + conf) / 2.0


def random_orders(n: int, B: int, seed: int) -> np.ndarray:
    """(B, n) uint8, each row a uniform random permutation (position -> node)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.stack([rng.permutation(n) for _ in range(B)]).astype(np.uint8) if B else \
        np.zeros((0, n), np.uint8)


# Workloads shaped like the paper's: Table III sweeps 13..60 nodes at a parent limit of 4
# (Sec. VI); Sec. VI's accuracy study uses a 20-node network with 1,000 samples.
WORKLOADS = {
    # tiny: 6 binary nodes, in-degree <= 2, 100 samples, k = 2, no prior
    "n6_k2_m100": dict(n=6, arity=2, max_indeg=2, m=100, k=2, prior=None, seed_index=0),
    # 20 ternary nodes, in-degree <= 3, 1000 samples, k = 4, 10%/10% pairwise prior
    "n20_k4_m1000": dict(n=20, arity=3, max_indeg=3, m=1000, k=4, prior=(0.1, 0.1), seed_index=1),
    # 40 ternary nodes, 2000 samples, k = 4
    "n40_k4_m2000": dict(n=40, arity=3, max_indeg=3, m=2000, k=4, prior=None, seed_index=2),
    # 40 ternary nodes, 1000 samples, k = 4 (fewer surviving parent sets than with 2000)
    "n40_k4_m1000": dict(n=40, arity=3, max_indeg=3, m=1000, k=4, prior=None, seed_index=5),
    # 60 ternary nodes, 1000 samples, k = 4 (the paper's largest graph)
    "n60_k4_m1000": dict(n=60, arity=3, max_indeg=3, m=1000, k=4, prior=None, seed_index=3),
}


def workload(name: str, seed_offset: int = 0):
    """Returns (data (m,n) uint8, arity (n,) uint8, k, R (n,n) float64 or None, net)."""
    w = WORKLOADS[name]
    seed = 0xB4E50000 + w["seed_index"] + 1000 * seed_offset
    net = random_network(w["n"], w["max_indeg"], w["arity"], seed)
    data = forward_sample(net, w["m"], seed + 1)
    R = None
    if w["prior"] is not None:
        R = prior_matrix(net, w["prior"][0], w["prior"][1], seed + 2)
    return data, net.arity.copy(), w["k"], R, net


def mlp_init_weights(n: int, d: int, H: int, seed: int) -> dict:
    """Seeded initial weights of the swap-proposal network (uniform, fan-in scaled,
    zero biases): E n x d, W1 H x (n d), W2 H x H, W3 P x H with P = n(n-1)/2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P = n * (n - 1) // 2
    return dict(
        E=rng.uniform(-1, 1, (n, d)).astype(np.float32),
        W1=(rng.uniform(-1, 1, (H, n * d)) / math.sqrt(n * d)).astype(np.float32),
        b1=np.zeros(H, np.float32),
        W2=(rng.uniform(-1, 1, (H, H)) / math.sqrt(H)).astype(np.float32),
        b2=np.zeros(H, np.float32),
        W3=(rng.uniform(-1, 1, (P, H)) / math.sqrt(H)).astype(np.float32),
        b3=np.zeros(P, np.float32),
    )


def uneven_batch(count: int, seed: int):
    """Many networks of uneven size: n ~ U{10..60}, per-node arity ~ U{2,3,4},
    m log-uniform in [200, 5000], k in {3, 4}, in-degree <= 3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for t in range(count):
        n = int(rng.integers(10, 61))
        ar = rng.integers(2, 5, size=n).astype(np.uint8)
        m = int(round(math.exp(rng.uniform(math.log(200), math.log(5000)))))
        k = int(rng.integers(3, 5))
        s = int(rng.integers(0, 2**31))
        net = random_network(n, 3, ar, s)
        out.append((forward_sample(net, m, s + 1), ar, k, None, net))
    return out
