"""What the trained surrogate gains: on the 1521-point FP16 problem, a plain
run (seed 100) logs exact evaluations, the network is trained on them by the
library's own kernels, and a surrogate-screened run (seed 200, top 25% of the
candidates evaluated exactly) is compared with a plain run of the same seed.
The screened run must use >= 3x fewer exact evaluations and reach at least
the hypervolume the plain run had reached with that many exact evaluations,
and come within 5% of the plain run's final hypervolume (this short run; the
benchmark's 200-generation run is held to 1%)."""

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def test_surrogate_screen_gains_over_plain():
    from paper_2303_04873_gb300 import build
    build.build()
    from paper_2303_04873_gb300 import ea, morea
    import bench
    p = synth.make_c2()
    gp = morea.Problem(p, max_changed=32)
    step = bench.local_step(p)
    orders = ea.bfs_orders(p.tets, p.n_points, 32)
    G, R = 30, 2
    log = []
    ea.run(gp, p, G, R, seed=100, step_scale=step, log=log, orders=orders, hv_every=G)
    feats = torch.cat([f for f, _ in log])
    targ = np.concatenate([o for _, o in log])
    net = morea.Mlp(3 * p.n_points, 512, 256, 3, max_batch=1024, seed=0)
    tr = ea.train_surrogate(net, feats, targ, epochs=10)
    assert np.all(tr["r2"] > 0.5), tr["r2"]
    del feats
    plain = ea.run(gp, p, G, R, seed=200, step_scale=step, orders=orders, hv_every=5)
    sur = ea.run(gp, p, G, R, seed=200, step_scale=step, orders=orders, hv_every=5, surrogate=tr["surrogate"],
                 ref=plain["ref"])
    assert plain["exact"] >= 3 * sur["exact"]
    hx = np.array([h[1] for h in plain["history"]], float)
    hv = np.array([h[2] for h in plain["history"]], float)
    assert sur["hv"] >= np.interp(sur["exact"], hx, hv)
    assert sur["hv"] >= 0.95 * plain["hv"]
