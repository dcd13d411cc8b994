"""Pins of the proposal-network oracle (oracle/mlp.py): rounding, a hand-worked forward
pass, finite-difference gradients, the mixture proposal and the Adam step."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import mlp


def test_bf16_round_against_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(5000) * 10 ** rng.uniform(-5, 5, 5000),
                        [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 65504.0, 3.0e38, 1e-40]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)
    assert mlp.bf16_round(1.0 + 2 ** -8) == 1.0                  # tie to even
    assert mlp.bf16_round(1.0 + 3 * 2 ** -9) == 1.0078125


def _hand_params():
    # n = 3 nodes, d = 1, H = 3, P = 3
    E = np.array([[1.0], [2.0], [3.0]])
    W1 = np.eye(3)
    b1 = np.array([-1.5, 0.0, -2.5])
    W2 = np.array([[1.0, 1.0, 0.0], [0.0, 0.0, 1.0], [1.0, 0.0, 0.0]])
    b2 = np.zeros(3)
    W3 = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0], [1.0, 1.0, 1.0]])
    b3 = np.array([0.0, 0.0, 0.5])
    return mlp.MLPParams(E, W1, b1, W2, b2, W3, b3)


def test_hand_worked_forward():
    """order (2, 0, 1): x = (E[2], E[0], E[1]) = (3, 1, 2); z1 = x + b1 = (1.5, 1, -0.5);
    h1 = (1.5, 1, 0); z2 = W2 h1 = (2.5, 0, 1.5) = h2; logits = W3 h2 + b3 = (2.5, 1.5, 4.5)."""
    f = mlp.mlp_forward(_hand_params(), np.array([[2, 0, 1]]))
    assert np.array_equal(f["x"][0], [3.0, 1.0, 2.0])
    assert np.array_equal(f["h1"][0], [1.5, 1.0, 0.0])
    assert np.array_equal(f["h2"][0], [2.5, 0.0, 1.5])
    assert np.array_equal(f["logits"][0], [2.5, 1.5, 4.5])
    # the mixture proposal: eps = 0 is log-softmax; eps = 1 is uniform
    lq0 = mlp.mlp_log_q(f["logits"], 0.0)[0]
    e = np.exp([2.5, 1.5, 4.5])
    assert np.allclose(lq0, np.log(e / e.sum()), rtol=1e-15)
    assert np.allclose(mlp.mlp_log_q(f["logits"], 1.0), np.log(1 / 3), rtol=1e-15)
    lq = mlp.mlp_log_q(f["logits"], 0.1)[0]
    assert np.allclose(np.exp(lq), 0.9 * e / e.sum() + 0.1 / 3, rtol=1e-14)


def test_hand_worked_gradient():
    """one sample, pair 2, target 1: d loss / d logit = sigmoid(4.5) - 1; only row 2 of W3
    and b3[2] receive it; dh2 = g * W3[2] = g (1, 1, 1), masked by z2 > 0 -> (g, 0, g)."""
    prm = _hand_params()
    loss, g = mlp.mlp_loss_grad(prm, np.array([[2, 0, 1]]), np.array([2]), np.array([1.0]))
    s = 1 / (1 + np.exp(-4.5))
    assert loss == pytest.approx(-np.log(s), rel=1e-12)
    gl = s - 1.0
    assert np.allclose(g["b3"], [0, 0, gl])
    assert np.allclose(g["W3"][2], gl * np.array([2.5, 0.0, 1.5])) and not g["W3"][:2].any()
    assert np.allclose(g["b2"], [gl, 0.0, gl], rtol=1e-2)       # bf16-rounded dz2


@pytest.mark.parametrize("seed", [0, 1])
def test_finite_difference_gradients(seed):
    rng = np.random.default_rng(seed)
    n, d, H, B = 5, 3, 6, 7
    prm = mlp.mlp_init(n, d, H, seed)
    prm.b1 = rng.standard_normal(H) * 0.3
    prm.b2 = rng.standard_normal(H) * 0.3
    prm.b3 = rng.standard_normal(n * (n - 1) // 2) * 0.3
    orders = np.stack([rng.permutation(n) for _ in range(B)])
    pairs = rng.integers(0, n * (n - 1) // 2, B)
    alpha = rng.uniform(0, 1, B)
    loss, g = mlp.mlp_loss_grad(prm, orders, pairs, alpha, rounded=False)
    h = 1e-6
    for name in ["E", "W1", "b1", "W2", "b2", "W3", "b3"]:
        arr = getattr(prm, name)
        flat = arr.reshape(-1)
        for idx in rng.choice(flat.size, min(flat.size, 12), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = mlp.mlp_loss_grad(prm, orders, pairs, alpha, rounded=False)
            flat[idx] = old - h
            lm, _ = mlp.mlp_loss_grad(prm, orders, pairs, alpha, rounded=False)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert g[name].reshape(-1)[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), name


def test_pair_index_matches_decode():
    for n in (2, 5, 60):
        for i, (a, b) in enumerate(itertools.combinations(range(n), 2)):
            assert mlp.pair_index(n, a, b) == i
            if n < 60 or i % 97 == 0:
                assert oracle.pair_decode(n, i) == (a, b)


def test_adam_first_step_closed_form():
    # after one step from zero moments the update is lr * g / (|g| + eps') elementwise
    prm = mlp.MLPParams(*(np.zeros(s) for s in [(2, 2), (3, 4), 3, (3, 3), 3, (1, 3), 1]))
    g = {k: np.full_like(getattr(prm, k), v) for k, v in zip(["E", "W1", "b1", "W2", "b2", "W3", "b3"],
                                                             [0.5, -2.0, 1e-3, 3.0, -1.0, 0.25, -4.0])}
    st = {}
    mlp.adam_step(prm, g, st, lr=0.01)
    for k in g:
        gv = g[k].reshape(-1)[0]
        assert getattr(prm, k).reshape(-1)[0] == pytest.approx(-0.01 * gv / (abs(gv) + 1e-8), rel=1e-9)
