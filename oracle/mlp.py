"""Oracle of the learned swap proposal (TEST INFRASTRUCTURE ONLY).

The paper proposes a new order by swapping two uniformly chosen nodes (Sec. III.C); it
has no learned proposal.  The proposal network here is defined by the build's own
specification and checked the same way as the rest: a plain FP64 numpy restatement with
the kernels' rounding points, pinned by hand-worked values and finite differences.

Network (positions p = 0..n-1, order sigma: position -> node, d-dimensional node
embeddings E, P = n(n-1)/2 swap pairs (a < b) in lexicographic order):
    x      = concat_p E[sigma(p)]                        (n*d)
    z1     = W1 x + b1,  h1 = relu(z1)                   (H)
    z2     = W2 h1 + b2, h2 = relu(z2)                   (H)
    logits = W3 h2 + b3                                  (P)
    q(pair | sigma) = (1 - eps) softmax(logits)[pair] + eps / P
Rounding points (``rounded=True``): weights, E and the GEMM inputs x, h1, h2 (and the
backward GEMM inputs dz2, dz1) are rounded to bfloat16 (round to nearest even); every
sum is FP64 here (FP32 accumulation in the kernels).

Training target: for a logged step (sigma, pair, delta) of the uniform-swap sampler, the
logit of the pair is fitted by binary cross-entropy to alpha = min(1, 10^delta), the
acceptance probability of that swap.  Loss = mean over the batch.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["bf16_round", "MLPParams", "mlp_init", "mlp_forward", "mlp_log_q", "mlp_loss_grad",
           "pair_index", "adam_step"]


def bf16_round(x):
    """Round float values to the nearest bfloat16 (ties to even), returned as float64.
    Works on the float32 bit pattern: add 0x7FFF plus the lowest kept bit, truncate."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


class MLPParams:
    def __init__(self, E, W1, b1, W2, b2, W3, b3):
        self.E, self.W1, self.b1, self.W2, self.b2, self.W3, self.b3 = E, W1, b1, W2, b2, W3, b3

    def copy(self):
        return MLPParams(*(np.array(a, np.float64) for a in self.arrays()))

    def arrays(self):
        return [self.E, self.W1, self.b1, self.W2, self.b2, self.W3, self.b3]


def mlp_init(n, d, H, seed):
    """Seeded initial parameters (uniform fan-in scaling), float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P = n * (n - 1) // 2
    E = rng.uniform(-1, 1, (n, d))
    W1 = rng.uniform(-1, 1, (H, n * d)) / math.sqrt(n * d)
    W2 = rng.uniform(-1, 1, (H, H)) / math.sqrt(H)
    W3 = rng.uniform(-1, 1, (P, H)) / math.sqrt(H)
    return MLPParams(E, W1, np.zeros(H), W2, np.zeros(H), W3, np.zeros(P))


def pair_index(n, a, b):
    """Lexicographic index of the position pair a < b."""
    return a * (2 * n - a - 1) // 2 + (b - a - 1)


def _r(x, rounded):
    return bf16_round(x) if rounded else np.asarray(x, np.float64)


def mlp_forward(prm: MLPParams, orders, rounded=True):
    """Forward pass for a batch of orders (B, n).  Returns a dict with the activations
    the backward pass needs and the logits (B, P)."""
    orders = np.asarray(orders, np.int64)
    E, W1, W2, W3 = (_r(a, rounded) for a in (prm.E, prm.W1, prm.W2, prm.W3))
    x = E[orders].reshape(orders.shape[0], -1)                 # concat over positions
    z1 = x @ W1.T + prm.b1
    h1 = _r(np.maximum(z1, 0.0), rounded)
    z2 = h1 @ W2.T + prm.b2
    h2 = _r(np.maximum(z2, 0.0), rounded)
    logits = h2 @ W3.T + prm.b3
    return dict(x=x, z1=z1, h1=h1, z2=z2, h2=h2, logits=logits, W1=W1, W2=W2, W3=W3)


def mlp_log_q(logits, eps):
    """log of the mixture proposal (1 - eps) softmax + eps / P, per row."""
    logits = np.asarray(logits, np.float64)
    P = logits.shape[-1]
    m = logits.max(axis=-1, keepdims=True)
    lse = m + np.log(np.exp(logits - m).sum(axis=-1, keepdims=True))
    return np.log((1.0 - eps) * np.exp(logits - lse) + eps / P)


def mlp_loss_grad(prm: MLPParams, orders, pairs, alpha, rounded=True, with_terms=False):
    """Mean BCE of sigmoid(logit[pair]) against alpha, and its gradient with respect to
    every parameter (dict with the same names).  with_terms: also the per-example
    factors every gradient sums over the batch, as grads["terms"]: the input x and the
    activations h1, h2, d loss / d logit[pair] ("dl"), the backward GEMM inputs dz2, dz1,
    the input gradient dx (B x n d, whose slices the embedding gradient sums), the
    pre-activations z1, z2 and the rounded weights W1, W2 they were computed with."""
    f = mlp_forward(prm, orders, rounded)
    B = f["x"].shape[0]
    rows = np.arange(B)
    l = f["logits"][rows, pairs]
    s = 1.0 / (1.0 + np.exp(-l))
    eps = 1e-300
    loss = -np.mean(alpha * np.log(s + eps) + (1 - alpha) * np.log(1 - s + eps))
    dl = (s - alpha) / B                                        # d loss / d logit[pair]
    dW3 = np.zeros_like(prm.W3)
    np.add.at(dW3, pairs, dl[:, None] * f["h2"])
    db3 = np.zeros_like(prm.b3)
    np.add.at(db3, pairs, dl)
    dh2 = dl[:, None] * f["W3"][pairs]
    dz2 = _r(dh2 * (f["z2"] > 0), rounded)
    dW2 = dz2.T @ f["h1"]
    db2 = dz2.sum(0)
    dh1 = dz2 @ f["W2"]
    dz1 = _r(dh1 * (f["z1"] > 0), rounded)
    dW1 = dz1.T @ f["x"]
    db1 = dz1.sum(0)
    dx = dz1 @ f["W1"]
    n = prm.E.shape[0]
    d = prm.E.shape[1]
    dE = np.zeros_like(prm.E)
    np.add.at(dE, np.asarray(orders, np.int64).reshape(-1), dx.reshape(-1, d))
    grads = dict(E=dE, W1=dW1, b1=db1, W2=dW2, b2=db2, W3=dW3, b3=db3)
    if with_terms:
        grads["terms"] = dict(x=f["x"], h1=f["h1"], h2=f["h2"], dl=dl, dz2=dz2, dz1=dz1, dx=dx,
                              z1=f["z1"], z2=f["z2"], W1=f["W1"], W2=f["W2"], dh2=dh2, dh1=dh1)
    return loss, grads


def adam_step(prm: MLPParams, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba) on every parameter; ``state`` holds m, v, t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    names = ["E", "W1", "b1", "W2", "b2", "W3", "b3"]
    for name in names:
        g = grads[name]
        m = state.setdefault("m_" + name, np.zeros_like(g))
        v = state.setdefault("v_" + name, np.zeros_like(g))
        m[...] = beta1 * m + (1 - beta1) * g
        v[...] = beta2 * v + (1 - beta2) * g * g
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        p = getattr(prm, name)
        p -= lr * mh / (np.sqrt(vh) + eps)
    return prm
