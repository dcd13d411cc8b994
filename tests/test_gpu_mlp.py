"""GPU parity of the proposal network's tensor-core kernels.

- bn_gemm_bf16 (tcgen05, TMEM accumulator) against a plain PyTorch fp32 matmul of the
  same bf16 operands: FP32 accumulation in a different order, so rtol 1e-4.
- forward, gradients and the Adam step against the FP64 oracle evaluated on the same
  bf16 rounding points: differences come from FP32 accumulation and from bf16 roundings
  of activations that land on the other side of a rounding boundary, so the bar is
  1e-2 of the tensor's max-norm per element and 1e-3 on the relative Frobenius norm."""
import numpy as np
import pytest

import synth
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def _weights(n, d, H, seed):
    w = synth.mlp_init_weights(n, d, H, seed)
    return w, omlp.MLPParams(*(np.asarray(w[k], np.float64) for k in ["E", "W1", "b1", "W2", "b2", "W3", "b3"]))


# gradient bars: 1e-2 of the tensor's max-norm per element, 1e-3 on the relative
# Frobenius norm of the difference
GRAD_ELEM, GRAD_NORM = 1e-2, 1e-3


def _close(a, b, elem=1e-2, norm=1e-3):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = max(np.abs(b).max(), 1e-30)
    assert np.abs(a - b).max() <= elem * scale, (np.abs(a - b).max(), scale)
    assert np.linalg.norm(a - b) <= norm * max(np.linalg.norm(b), 1e-30) + 1e-30


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 512, 1920), (384, 256, 192), (256, 1792, 512),
                                   (512, 512, 256)])
def test_gemm_matches_torch(gpu, M, N, K):
    import torch
    g = torch.Generator().manual_seed(M * 7 + N + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    ref = A.float() @ B.float().T
    out = gpu.gemm_bf16(A.cuda(), B.cuda()).cpu()
    torch.testing.assert_close(out, ref, rtol=1e-4, atol=1e-3)


def test_gemm_identity_and_zero_k(gpu):
    import torch
    A = torch.zeros(128, 64, dtype=torch.bfloat16)
    A[:, :64] = torch.eye(128)[:, :64].to(torch.bfloat16)
    B = torch.arange(128 * 64, dtype=torch.float32).reshape(128, 64).remainder(7).to(torch.bfloat16)
    out = gpu.gemm_bf16(A.cuda(), B.cuda()).cpu()
    # C[i][j] = sum_k A[i][k] B[j][k] = B[j][i] for i < 64
    assert torch.equal(out[:64], B.float().T[:64])
    assert torch.equal(out[64:], torch.zeros(64, 128))


@pytest.mark.parametrize("n,d,H,B", [(6, 8, 128, 40), (60, 32, 512, 256)])
def test_forward_matches_oracle(gpu, n, d, H, B):
    w, prm = _weights(n, d, H, 5)
    net = gpu.mlp_create(n, w, hidden=H, d=d, batch_cap=B)
    orders = synth.random_orders(n, B, 6)
    logits = gpu.mlp_forward(net, orders)
    ref = omlp.mlp_forward(prm, orders)["logits"]
    _close(logits, ref)


@pytest.mark.parametrize("n,d,H,B", [(6, 8, 128, 40), (60, 32, 512, 256)])
def test_gradients_and_adam_match_oracle(gpu, n, d, H, B):
    w, prm = _weights(n, d, H, 9)
    net = gpu.mlp_create(n, w, hidden=H, d=d, batch_cap=B, lr=1e-3)
    rng = np.random.default_rng(n)
    orders = synth.random_orders(n, B, 10)
    pairs = rng.integers(0, n * (n - 1) // 2, B).astype(np.uint32)
    alpha = rng.uniform(0, 1, B).astype(np.float32)
    loss = gpu.mlp_loss_grad(net, orders, pairs, alpha)
    ref_loss, ref_g = omlp.mlp_loss_grad(prm, orders, pairs.astype(np.int64), alpha.astype(np.float64),
                                         with_terms=True)
    assert loss == pytest.approx(ref_loss, rel=1e-4)
    # Every gradient is a sum over the batch of per-example terms of either sign, so its
    # rounding error scales with the sum of the terms' magnitudes (the usual bound for a
    # floating-point sum), not with the sum itself when terms cancel: the norm bar is
    # taken relative to that magnitude sum, from the oracle's per-example factors.
    T = {key: np.abs(v) for key, v in ref_g["terms"].items()}
    pr = pairs.astype(np.int64)
    mag = {"W1": T["dz1"].T @ T["x"], "b1": T["dz1"].sum(0), "W2": T["dz2"].T @ T["h1"], "b2": T["dz2"].sum(0),
           "W3": np.zeros_like(ref_g["W3"]), "b3": np.zeros_like(ref_g["b3"]), "E": np.zeros_like(ref_g["E"])}
    np.add.at(mag["W3"], pr, T["dl"][:, None] * T["h2"])
    np.add.at(mag["b3"], pr, T["dl"])
    np.add.at(mag["E"], np.asarray(orders, np.int64).reshape(-1), T["dx"].reshape(-1, d))
    # ReLU decisions the kernels take in FP32 and the oracle in FP64: the kernels' sums
    # differ from the oracle's by FP32 accumulation (K 2^-24 of the terms' magnitude sum,
    # at most 2^-13 for K <= 2048) and, for layer 2, by layer-1 outputs whose bf16 rounding
    # fell the other way (each one ulp, 2^-8 of its term; measured up to 4e-5 of the sum).
    # A pre-activation within 2^-13 of its magnitude sum of zero may therefore fall on
    # either side, and then the term it gates in the weight and bias gradients is present
    # on one side only.  Either is valid: the element bar grows by those terms'
    # magnitudes (first order).
    tau = 2.0 ** -13
    near1 = np.abs(ref_g["terms"]["z1"]) <= tau * (T["x"] @ T["W1"].T + np.abs(w["b1"]))
    near2 = np.abs(ref_g["terms"]["z2"]) <= tau * (T["h1"] @ T["W2"].T + np.abs(w["b2"]))
    assert near1.mean() < 1e-2 and near2.mean() < 1e-2, (near1.sum(), near2.sum())
    g1 = near1 * T["dh1"]
    g2 = near2 * T["dh2"]
    extra = {"W1": g1.T @ T["x"], "b1": g1.sum(0), "W2": g2.T @ T["h1"], "b2": g2.sum(0)}
    for name in ["E", "W1", "b1", "W2", "b2", "W3", "b3"]:
        g = gpu.mlp_read(net, name, grad=True).astype(np.float64)
        ref = ref_g[name]
        bound = GRAD_ELEM * np.abs(ref).max() + extra.get(name, 0.0)
        assert (np.abs(g - ref) <= bound).all(), (name, (np.abs(g - ref) - bound).max())
        assert np.linalg.norm(g - ref) <= GRAD_NORM * np.linalg.norm(mag[name]), name
    lr, eps = 1e-3, 1e-8
    gpu.mlp_adam_step(net)
    for name in ["E", "W1", "b1", "W2", "b2", "W3", "b3"]:
        before = np.asarray(w[name], np.float32)
        upd = gpu.mlp_read(net, name).astype(np.float64) - before.astype(np.float64)
        # Adam's first step (m, v from zero, bias-corrected) is -lr g / (|g| + eps), a
        # monotone function of g.  The gradient check above bounds every element of the
        # kernel's gradient within delta (its element bar) of the oracle's, so each update
        # must lie between
        # the steps of g_ref - delta and g_ref + delta -- a tight bound wherever
        # |g_ref| >> delta, and one that admits either sign only where it is within delta
        # of zero.  Slack: FP32 rounding of the step and of the updated weight.
        g = ref_g[name]
        delta = GRAD_ELEM * np.abs(g).max() + extra.get(name, 0.0)
        step = lambda x: -lr * x / (np.abs(x) + eps)            # noqa: E731
        lo, hi = step(g + delta), step(g - delta)
        slack = 1e-6 * lr + 2.0 * np.spacing(np.abs(before)).astype(np.float64)
        assert (upd >= lo - slack).all() and (upd <= hi + slack).all(), name
        clear = np.abs(g) > 2 * delta
        assert np.array_equal(np.sign(upd[clear]), -np.sign(g[clear])), name
        assert np.abs(upd).max() <= lr * (1 + 1e-6) + slack.max(), name     # |first step| <= lr


def test_batch_above_capacity_rejected(gpu):
    w, _ = _weights(6, 8, 128, 1)
    net = gpu.mlp_create(6, w, hidden=128, d=8, batch_cap=100)
    with pytest.raises(gpu.BNError) as e:
        gpu.mlp_forward(net, synth.random_orders(6, 129, 1))
    assert e.value.code == gpu.EINVAL


def test_training_steps_are_deterministic(gpu):
    """Gradients are summed in a fixed order (no floating-point atomics): two networks
    trained on the same batches hold the same bits, including batches that repeat a pair."""
    n, d, H, B = 20, 16, 128, 200
    w, _ = _weights(n, d, H, 4)
    nets = [gpu.mlp_create(n, w, hidden=H, d=d, batch_cap=B, lr=2e-3) for _ in range(2)]
    rng = np.random.default_rng(8)
    for step in range(3):
        orders = synth.random_orders(n, B, 30 + step)
        pairs = rng.integers(0, 12, B).astype(np.uint32)          # few distinct pairs: many repeats
        alpha = rng.uniform(0, 1, B).astype(np.float32)
        losses = [gpu.mlp_loss_grad(net, orders, pairs, alpha) for net in nets]
        assert losses[0] == losses[1]
        for net in nets:
            gpu.mlp_adam_step(net)
    for name in ["E", "W1", "b1", "W2", "b2", "W3", "b3"]:
        assert np.array_equal(gpu.mlp_read(nets[0], name), gpu.mlp_read(nets[1], name)), name
        assert np.array_equal(gpu.mlp_read(nets[0], name, grad=True), gpu.mlp_read(nets[1], name, grad=True)), name
