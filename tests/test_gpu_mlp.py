"""Surrogate network kernels (tcgen05 tensor-core products, backward, Adam)
against the FP64 oracle of oracle/mlp.py with the same bfloat16-rounded
operands, element by element.

Error model (BF16 storage, FP32 accumulation).  Every product C = A B of the
network takes its operands exactly as the oracle has them until an operand
is itself a result stored in BF16 (h1, h2, dh2, dh1).  ``mlp_bounds``
carries an error scale E through the forward and backward pass with the
oracle's values:
- a stored result adds one BF16 rounding, u |value| (u = 2^-8, the unit
  roundoff), to its inherited error;
- a product propagates its operands' errors; roundings are independent and
  unbiased, so they combine in quadrature, E_C = sqrt(E_A^2 B^2 + A^2 E_B^2)
  (element-wise squares, matrix products);
- FP32 accumulation over K terms adds 2^-24 (sqrt(K) sqrt(A^2 B^2) +
  K/8 |A| |B|)_ij: independent roundings plus a linear part for an
  accumulator that truncates;
- a ReLU is exact where the oracle's pre-activation is below -LAMBDA E and
  1-Lipschitz elsewhere; where |pre-activation| <= LAMBDA E the GPU's mask
  may differ, so the masked gradient may take its whole unmasked value.
Every output and gradient element must satisfy |gpu - oracle| <= LAMBDA E
with LAMBDA = 8.  A wrong row, column or bias element is off by the size of
the values themselves, far outside that band.
One Adam step is compared within 1e-5 relative of the oracle's update from
the same gradients."""

import numpy as np
import pytest
import torch

import synth
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8
LAMBDA = 8.0


@pytest.fixture(scope="module")
def mo():
    from paper_2303_04873_gb300 import build
    build.build()
    from paper_2303_04873_gb300 import morea
    return morea


def _acc(A, B):
    """FP32 accumulation error of A @ B over K = A.shape[1] terms: independent
    roundings in quadrature, 2^-24 sqrt(K) sqrt(A^2 B^2), plus a linear part
    (K / 8) 2^-24 (|A| |B|) for an accumulator that truncates (the tensor
    cores sum each 16-term block before adding it)."""
    K = A.shape[1]
    return 2.0 ** -24 * (np.sqrt(K) * np.sqrt((A ** 2) @ (B ** 2)) + K / 8.0 * (np.abs(A) @ np.abs(B)))


def _prod_err(EA, B, A, EB):
    """Quadrature error of A @ B from operand errors EA (of A) and EB (of B)."""
    return np.sqrt((EA ** 2) @ (B ** 2) + (A ** 2) @ (EB ** 2))


def _relu_err(z, Ez, h):
    """Error of the stored activation h = bf16(relu(z)) given z's error."""
    return np.where(z < -LAMBDA * Ez, 0.0, np.sqrt(Ez ** 2 + (U_BF16 * h) ** 2))


def _masked_err(z, Ez, pre, Epre, d):
    """Error of the stored gradient d = bf16(pre * (z > 0))."""
    open_mask = np.abs(z) <= LAMBDA * Ez
    inside = np.where(z > 0, np.sqrt(Epre ** 2 + (U_BF16 * d) ** 2), 0.0)
    return np.where(open_mask, (np.abs(pre) + LAMBDA * Epre) / LAMBDA, inside)


def mlp_bounds(P, x, t):
    """Element-wise error scales E of the GPU's y and gradients (see the
    module docstring); the test allows LAMBDA E."""
    q = omlp.bf16_round
    W1, b1, W2, b2, W3, b3 = P
    X, W1q, W2q, W3q = q(x), q(W1), q(W2), q(W3)
    A = np.abs
    z1 = X @ W1q.T + b1
    h1 = q(np.maximum(z1, 0.0))
    z2 = h1 @ W2q.T + b2
    h2 = q(np.maximum(z2, 0.0))
    y = h2 @ W3q.T + b3
    n, m = y.shape
    Z = np.zeros_like
    E_z1 = _acc(X, W1q.T) + 2.0 ** -24 * A(b1)
    E_h1 = _relu_err(z1, E_z1, h1)
    E_z2 = _prod_err(E_h1, W2q.T, h1, Z(W2q.T)) + _acc(h1, W2q.T) + 2.0 ** -24 * A(b2)
    E_h2 = _relu_err(z2, E_z2, h2)
    E_y = _prod_err(E_h2, W3q.T, h2, Z(W3q.T)) + _acc(h2, W3q.T) + 2.0 ** -24 * A(b3)
    dy = 2.0 * (y - np.asarray(t, np.float64)) / (n * m)
    E_dy = 2.0 * E_y / (n * m) + 2.0 ** -23 * A(dy)
    ones = np.ones((1, n))
    E_gW3 = _prod_err(E_dy.T, h2, dy.T, E_h2) + _acc(dy.T, h2)
    E_gb3 = np.sqrt((E_dy ** 2).sum(0)) + _acc(ones, dy)[0]
    pre2 = dy @ W3q
    E_pre2 = _prod_err(E_dy, W3q, dy, Z(W3q)) + _acc(dy, W3q)
    dh2 = q(pre2 * (h2 > 0))
    E_dh2 = _masked_err(z2, E_z2, pre2, E_pre2, dh2)
    E_gW2 = _prod_err(E_dh2.T, h1, dh2.T, E_h1) + _acc(dh2.T, h1)
    E_gb2 = np.sqrt((E_dh2 ** 2).sum(0)) + _acc(ones, dh2)[0]
    pre1 = dh2 @ W2q
    E_pre1 = _prod_err(E_dh2, W2q, dh2, Z(W2q)) + _acc(dh2, W2q)
    dh1 = q(pre1 * (h1 > 0))
    E_dh1 = _masked_err(z1, E_z1, pre1, E_pre1, dh1)
    E_gW1 = _prod_err(E_dh1.T, X, dh1.T, Z(X)) + _acc(dh1.T, X)
    E_gb1 = np.sqrt((E_dh1 ** 2).sum(0)) + _acc(ones, dh1)[0]
    return E_y, (E_gW1, E_gb1, E_gW2, E_gb2, E_gW3, E_gb3)


def assert_within(got, want, scale, what):
    got = np.asarray(got, np.float64)
    err = np.abs(got - want)
    bound = LAMBDA * scale
    bad = err > bound
    assert not bad.any(), (f"{what}: {int(bad.sum())} of {bad.size} elements outside the bound; worst excess "
                           f"{float((err - bound).max()):.3e} at {np.unravel_index(np.argmax(err - bound), err.shape)}")


@pytest.mark.parametrize("n_in,h1,h2,n_out,batch", [(4563, 512, 256, 3, 1024), (37, 64, 128, 5, 50),
                                                     (130, 128, 64, 1, 129)])
def test_forward_and_gradients_match_oracle(mo, n_in, h1, h2, n_out, batch):
    net = mo.Mlp(n_in, h1, h2, n_out, max_batch=batch, seed=1)
    rng = np.random.default_rng(2)
    params = net.get_params()
    x = rng.normal(0, 1.0, size=(batch, n_in)).astype(np.float32)
    t = rng.normal(0, 1.0, size=(batch, n_out)).astype(np.float32)
    X = torch.as_tensor(x).cuda()
    Tt = torch.as_tensor(t).cuda()
    y = net.forward(X).cpu().numpy()
    g, loss = net.gradients(X, Tt)
    g = g.cpu().numpy()
    P = omlp.split(params, n_in, net.kin, h1, h2, n_out)
    P = tuple(np.asarray(p, np.float64) for p in P)
    yo, lo, go = omlp.forward(P, x, t, bf16=True)
    E_y, E_g = mlp_bounds(P, x, t)
    assert_within(y, yo, E_y, "forward output")
    assert float(loss.item()) == pytest.approx(lo, rel=1e-2)
    gg = omlp.split(g, n_in, net.kin, h1, h2, n_out)
    names = ("dW1", "db1", "dW2", "db2", "dW3", "db3")
    for name, a, b, e in zip(names, gg, go, E_g):
        assert_within(a, b, e, name)
    # padded input columns get no gradient
    W1g = g[:h1 * net.kin].reshape(h1, net.kin)
    assert np.all(W1g[:, n_in:] == 0.0)
    # every wait inside the tensor-core products completed
    assert net.device_status() == 0


def test_adam_step_matches_oracle(mo):
    net = mo.Mlp(200, 128, 64, 3, max_batch=256, seed=3)
    rng = np.random.default_rng(4)
    X = torch.as_tensor(rng.normal(size=(256, 200)).astype(np.float32)).cuda()
    T = torch.as_tensor(rng.normal(size=(256, 3)).astype(np.float32)).cuda()
    w0 = net.get_params().astype(np.float64)
    g, _ = net.gradients(X, T)
    g = g.cpu().numpy().astype(np.float64)
    net.train_step(X, T, lr=1e-3)
    w1 = net.get_params()
    want, _, _ = omlp.adam_step(w0, g, np.zeros_like(w0), np.zeros_like(w0), 1, lr=1e-3)
    np.testing.assert_allclose(w1, want, rtol=1e-5, atol=1e-7)


def test_training_fits_a_teacher(mo):
    rng = np.random.default_rng(5)
    n_in, n = 300, 4096
    teacher = mo.Mlp(n_in, 64, 64, 3, max_batch=1024, seed=11)
    x = torch.as_tensor(rng.normal(size=(n, n_in)).astype(np.float32)).cuda()
    y = teacher.forward(x)
    y = (y - y.mean(0)) / y.std(0)
    net = mo.Mlp(n_in, 128, 64, 3, max_batch=1024, seed=12)
    first = None
    for it in range(400):
        a = (it * 1024) % n
        loss = float(net.train_step(x[a:a + 1024], y[a:a + 1024].contiguous(), lr=2e-3).item())
        first = first if first is not None else loss
    pred = net.forward(x)
    final = float(((pred - y) ** 2).mean().item())
    assert final < first / 10, (first, final)
    assert net.device_status() == 0 and teacher.device_status() == 0


def test_partial_features(mo):
    import oracle
    p = synth.make_c0(n_sol=4)
    gp = mo.Problem(p)
    gp.eval_full(torch.as_tensor(p.sol_src).cuda(), torch.as_tensor(p.sol_tgt).cuda())
    adj = synth.vertex_adjacency(p.tets, p.n_points)
    rd = synth.partial_requests(p, adj, 1, 4, 12, 1.0, 8)[0]
    dv = {k: torch.as_tensor(v).cuda() for k, v in rd.items()}
    f = gp.partial_features(dv["slot"], dv["chg_off"], dv["chg_pts"], dv["chg_src"], dv["chg_tgt"]).cpu().numpy()
    shape = (p.nx, p.ny, p.nz)
    snap = np.vectorize(lambda x, a: oracle.snap1(float(x), shape[a], 8))
    for r in range(4):
        s, t = p.sol_src[r].copy(), p.sol_tgt[r].copy()
        a, b = rd["chg_off"][r], rd["chg_off"][r + 1]
        s[rd["chg_pts"][a:b]] = rd["chg_src"][a:b]
        t[rd["chg_pts"][a:b]] = rd["chg_tgt"][a:b]
        ax = np.arange(3)[None, :]
        want = (snap(t, ax) - snap(s, ax)) / 256.0
        np.testing.assert_array_equal(f[r].reshape(-1, 3), want.astype(np.float32))
