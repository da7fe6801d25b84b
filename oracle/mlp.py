"""FP64 oracle of the surrogate network and its training step.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy: a 3-layer
perceptron x -> relu(x W1^T + b1) -> relu(. W2^T + b2) -> . W3^T + b3, the
mean squared error against targets, its gradient by the chain rule written
out layer by layer, and one Adam step.  ``bf16=True`` rounds the inputs,
weights and stored activations/gradients to bfloat16 (round to nearest
even) at the points where the GPU stores them in that format, so GPU results
can be compared against the same quantised operands.  Pinned in
tests/test_oracle_mlp.py by central finite differences and closed forms.
"""

from __future__ import annotations

import numpy as np


def bf16_round(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def split(params, n_in, kin, h1, h2, n_out):
    """Parameter vector (library layout) -> (W1 [h1][n_in], b1, W2, b2, W3, b3)."""
    p = np.asarray(params, np.float64)
    o = 0
    W1 = p[o:o + h1 * kin].reshape(h1, kin)[:, :n_in]
    o += h1 * kin
    b1 = p[o:o + h1]
    o += h1
    W2 = p[o:o + h2 * h1].reshape(h2, h1)
    o += h2 * h1
    b2 = p[o:o + h2]
    o += h2
    W3 = p[o:o + n_out * h2].reshape(n_out, h2)
    o += n_out * h2
    b3 = p[o:o + n_out]
    return W1, b1, W2, b2, W3, b3


def join(grads, n_in, kin, h1, h2, n_out):
    W1, b1, W2, b2, W3, b3 = grads
    W1p = np.zeros((h1, kin))
    W1p[:, :n_in] = W1
    return np.concatenate([W1p.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])


def forward(params, x, t=None, bf16=False):
    """Returns y and, if t is given, (loss, grads as a tuple of arrays)."""
    W1, b1, W2, b2, W3, b3 = params
    q = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    X, W1q, W2q, W3q = q(x), q(W1), q(W2), q(W3)
    z1 = X @ W1q.T + b1
    h1 = q(np.maximum(z1, 0.0))
    z2 = h1 @ W2q.T + b2
    h2 = q(np.maximum(z2, 0.0))
    y = h2 @ W3q.T + b3
    if t is None:
        return y
    n, m = y.shape
    d = y - np.asarray(t, np.float64)
    loss = float(np.mean(d * d))
    dy = 2.0 * d / (n * m)
    gW3 = dy.T @ h2
    gb3 = dy.sum(axis=0)
    dh2 = q((dy @ W3q) * (h2 > 0))
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(axis=0)
    dh1 = q((dh2 @ W2q) * (h1 > 0))
    gW1 = dh1.T @ X
    gb1 = dh1.sum(axis=0)
    return y, loss, (gW1, gb1, gW2, gb2, gW3, gb3)


def adam_step(w, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
