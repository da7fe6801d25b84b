"""Pins of the surrogate-network oracle (oracle/mlp.py): analytic gradients
against central finite differences in FP64, closed-form forward values,
hand-checked bfloat16 rounding, and the first Adam step's closed form."""

import numpy as np
import pytest

from oracle import mlp


def _net(rng, n_in=7, h1=6, h2=5, n_out=3):
    return (rng.normal(0, 0.5, (h1, n_in)), rng.normal(0, 0.1, h1), rng.normal(0, 0.5, (h2, h1)),
            rng.normal(0, 0.1, h2), rng.normal(0, 0.5, (n_out, h2)), rng.normal(0, 0.1, n_out))


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    params = _net(rng)
    x = rng.normal(size=(9, 7))
    t = rng.normal(size=(9, 3))
    _, loss, grads = mlp.forward(params, x, t)
    h = 1e-6
    for pi, (p, g) in enumerate(zip(params, grads)):
        flat = p.reshape(-1)
        num = np.zeros_like(flat)
        for i in range(flat.size):
            keep = flat[i]
            flat[i] = keep + h
            _, lp, _ = mlp.forward(params, x, t)
            flat[i] = keep - h
            _, lm, _ = mlp.forward(params, x, t)
            flat[i] = keep
            num[i] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(g.reshape(-1), num, rtol=1e-6, atol=1e-9, err_msg=f"param {pi}")


def test_forward_closed_form():
    # W1 = W2 = 0: h1 = relu(b1), h2 = relu(b2), y = W3 relu(b2) + b3 for every input
    n_in, h1, h2 = 4, 3, 2
    W3 = np.array([[1.0, -2.0], [0.5, 0.25], [3.0, 1.0]])
    b2 = np.array([2.0, -1.0])
    b3 = np.array([0.1, 0.2, 0.3])
    params = (np.zeros((h1, n_in)), np.ones(h1), np.zeros((h2, h1)), b2, W3, b3)
    y = mlp.forward(params, np.random.default_rng(1).normal(size=(5, n_in)))
    want = W3 @ np.array([2.0, 0.0]) + b3
    np.testing.assert_allclose(y, np.tile(want, (5, 1)), rtol=0, atol=1e-15)
    # loss gradient w.r.t. b3 is the mean residual times 2 / n_out
    t = np.zeros((5, 3))
    _, loss, g = mlp.forward(params, np.ones((5, n_in)), t)
    np.testing.assert_allclose(g[5], 2.0 * want / 3.0, rtol=1e-15)
    assert loss == pytest.approx(np.mean(want ** 2), rel=1e-15)


def test_bf16_rounding_by_hand_and_against_torch():
    # ties go to the even 8-bit mantissa: 1 + 2^-8 -> 1, 1 + 2^-7 + 2^-8 -> 1 + 2^-6
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 1.0 + 2 ** -7 + 2 ** -8, 0.0])
    want = np.array([1.0, 1.0, 1.0 + 2 ** -7, -2.5, 1.0 + 2 ** -6, 0.0])
    np.testing.assert_array_equal(mlp.bf16_round(vals), want)
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(3).normal(0, 100, 10000).astype(np.float32)
    ref = torch.from_numpy(r).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(r), ref)


def test_first_adam_step_closed_form():
    w = np.array([1.0, -1.0, 0.5])
    g = np.array([0.2, -3.0, 1e-3])
    w1, m, v = mlp.adam_step(w, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # m_hat = g, v_hat = g^2 -> update = lr * g / (|g| + eps)
    np.testing.assert_allclose(w1, w - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_layout_roundtrip():
    rng = np.random.default_rng(2)
    params = _net(rng, n_in=10)
    vec = mlp.join(params, 10, 64, 6, 5, 3)
    back = mlp.split(vec, 10, 64, 6, 5, 3)
    for a, b in zip(params, back):
        np.testing.assert_array_equal(a, b)
    assert vec.size == 6 * 64 + 6 + 5 * 6 + 5 + 3 * 5 + 3
