"""Surrogate network kernels (tcgen05 tensor-core products, backward, Adam)
against the FP64 oracle of oracle/mlp.py with the same bfloat16-rounded
operands.

Tolerances (BF16 storage, FP32 accumulation): forward outputs within 5e-3 of
the oracle in relative norm, each gradient block within 2e-2, one Adam step
within 1e-5 relative of the oracle's update from the same gradients."""

import numpy as np
import pytest
import torch

import synth
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mo():
    from paper_2303_04873_gb300 import build
    build.build()
    from paper_2303_04873_gb300 import morea
    return morea


def relnorm(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


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
    assert relnorm(y, yo) < 5e-3
    assert float(loss.item()) == pytest.approx(lo, rel=1e-2)
    gg = omlp.split(g, n_in, net.kin, h1, h2, n_out)
    for k, (a, b) in enumerate(zip(gg, go)):
        assert relnorm(a, b) < 2e-2, (k, relnorm(a, b))
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
