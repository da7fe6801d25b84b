"""Batched multi-problem evaluation, CUDA-graph replay, launch shapes and the
autotuner.  The per-problem results of a batch must be bit-identical to
per-problem morea_eval_full calls (same per-item arithmetic, same reduction
order) and must not depend on the launch shape; one batch member is also
checked against the FP64 oracle."""

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mo():
    from paper_2303_04873_gb300 import build
    build.build()
    from paper_2303_04873_gb300 import morea
    return morea


def _problems():
    out = []
    specs = [((24, 24, 24), (3, 3, 3), 6), ((20, 28, 16), (2, 4, 2), 3), ((32, 18, 22), (4, 2, 3), 9),
             ((17, 23, 29), (2, 3, 4), 4)]
    for m, (shape, cells, pop) in enumerate(specs):
        nx, ny, nz = shape
        ax = [np.linspace(-0.5, n - 0.5, c + 1) for n, c in zip(shape, cells)]
        ell = [(nx * 0.4, ny * 0.5, nz * 0.5, nx * 0.25, ny * 0.2, nz * 0.3, 60.0),
               (nx * 0.65, ny * 0.4, nz * 0.45, nx * 0.15, ny * 0.25, nz * 0.2, 120.0)]
        out.append(synth.make_problem(
            name=f"b{m}", shape_xyz=shape, ellipsoids=ell, background=0.0, amp=1.5, noise_sigma=4.0,
            dtype="f16", xs=ax[0], ys=ax[1], zs=ax[2], n_guid=40, n_sol=pop,
            jitter=0.15 * min(n / c for n, c in zip(shape, cells)), tissue=[1.0, 0.5, 3.0],
            seeds=(20 + m, 30 + m, 40 + m), trunc_radius=2.5))
    return out


def _full(gp, p):
    S = torch.as_tensor(p.sol_src).cuda()
    T = torch.as_tensor(p.sol_tgt).cuda()
    obj, fo, sev = gp.eval_full(S, T)
    torch.cuda.synchronize()
    return obj.cpu().numpy(), fo.cpu().numpy(), sev.cpu().numpy(), gp.read_records(p.n_solutions)


def test_batch_equals_per_problem_and_oracle(mo):
    probs = _problems()
    gps = [mo.Problem(p) for p in probs]
    ref = [_full(gp, p) for gp, p in zip(gps, probs)]
    batch = mo.Batch(gps)
    srcs = [torch.as_tensor(p.sol_src).cuda() for p in probs]
    tgts = [torch.as_tensor(p.sol_tgt).cuda() for p in probs]
    outs = batch.eval_full(srcs, tgts)
    torch.cuda.synchronize()
    for i, (p, gp) in enumerate(zip(probs, gps)):
        np.testing.assert_array_equal(outs[i][0].cpu().numpy(), ref[i][0])
        np.testing.assert_array_equal(outs[i][1].cpu().numpy(), ref[i][1])
        np.testing.assert_array_equal(outs[i][2].cpu().numpy(), ref[i][2])
        np.testing.assert_array_equal(gp.read_records(p.n_solutions), ref[i][3])
    p, gp = probs[2], gps[2]
    orc = oracle.Oracle(p, subvoxel_bits=gp.subvoxel_bits, trunc_radius=gp.trunc_radius)
    for s in (0, p.n_solutions - 1):
        r = orc.eval(p.sol_src[s], p.sol_tgt[s], with_tets=True)
        np.testing.assert_array_equal(ref[2][3][s]["n_vox"], r["tets"]["n_vox"])
        np.testing.assert_allclose(outs[2][0][s].cpu().numpy(), r["obj"], rtol=1e-5, atol=1e-10)


def test_graph_replay_reads_current_buffers(mo):
    probs = _problems()
    gps = [mo.Problem(p) for p in probs]
    batch = mo.Batch(gps)
    srcs = [torch.as_tensor(p.sol_src).cuda() for p in probs]
    tgts = [torch.as_tensor(p.sol_tgt).cuda() for p in probs]
    outs = mo.Batch.outputs(srcs)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.capture(srcs, tgts, outs, stream)
        batch.replay(stream)
    stream.synchronize()
    first = [o[0].clone() for o in outs]
    direct = batch.eval_full(srcs, tgts)
    torch.cuda.synchronize()
    for a, b in zip(first, direct):
        assert torch.equal(a, b[0])
    # new contents in the captured buffers, replay again
    for s, t in zip(srcs, tgts):
        s.copy_(torch.flip(s, dims=[0]))
        t.copy_(torch.flip(t, dims=[0]))
    with torch.cuda.stream(stream):
        batch.replay(stream)
    stream.synchronize()
    direct = batch.eval_full(srcs, tgts)
    torch.cuda.synchronize()
    for a, b, f in zip(outs, direct, first):
        assert torch.equal(a[0], b[0])
        assert torch.equal(a[0], torch.flip(f, dims=[0]))


@pytest.mark.parametrize("shape", [(4, 0), (16, 0), (8, 1), (8, 4), (2, 64)])
def test_results_do_not_depend_on_launch_shape(mo, shape):
    p = synth.make_c0(n_sol=8)
    gp = mo.Problem(p)
    base = _full(gp, p)
    adj = synth.vertex_adjacency(p.tets, p.n_points)
    rd = synth.partial_requests(p, adj, 1, 4, 32, 1.0, 5)[0]
    dv = {k: torch.as_tensor(v).cuda() for k, v in rd.items()}
    pb = gp.eval_partial(dv["slot"], dv["chg_off"], dv["chg_pts"], dv["chg_src"], dv["chg_tgt"])[0].cpu().numpy()
    gp.set_launch(*shape)
    again = _full(gp, p)
    pa = gp.eval_partial(dv["slot"], dv["chg_off"], dv["chg_pts"], dv["chg_src"], dv["chg_tgt"])[0].cpu().numpy()
    np.testing.assert_array_equal(again[0], base[0])
    np.testing.assert_array_equal(again[3], base[3])
    np.testing.assert_array_equal(pa, pb)
    with pytest.raises(mo.MoreaError):
        gp.set_launch(0, 0)


def test_autotuner_picks_and_caches(mo, tmp_path):
    from paper_2303_04873_gb300 import autotune
    probs = _problems()
    gps = [mo.Problem(p) for p in probs]
    batch = mo.Batch(gps)
    srcs = [torch.as_tensor(p.sol_src).cuda() for p in probs]
    tgts = [torch.as_tensor(p.sol_tgt).cuda() for p in probs]
    outs = mo.Batch.outputs(srcs)
    ref = [o[0].clone() for o in batch.eval_full(srcs, tgts)]
    key = autotune.signature(gps, [p.n_solutions for p in probs], "batch_full")
    path = str(tmp_path / "tune.json")
    bps, chunk, t = autotune.tune(batch, lambda: batch.eval_full(srcs, tgts, outs), key,
                                  candidates=[(4, 0), (8, 0), (8, 2)], reps=3, path=path)
    assert (bps, chunk) in t and len(t) == 3
    bps2, chunk2, t2 = autotune.tune(batch, lambda: batch.eval_full(srcs, tgts, outs), key, path=path)
    assert (bps2, chunk2) == (bps, chunk) and t2 == {}
    batch.eval_full(srcs, tgts, outs)
    torch.cuda.synchronize()
    for a, b in zip(outs, ref):
        assert torch.equal(a[0], b)


def test_batch_rejects_mixed_modes(mo):
    a = mo.Problem(synth.make_c0(n_sol=2))
    b = mo.Problem(synth.make_c0(n_sol=2), g_mode=2)
    with pytest.raises(mo.MoreaError):
        mo.Batch([a, b])
    with pytest.raises(mo.MoreaError):
        mo.Batch([a, a])


def test_batch_latency_per_problem(mo):
    """The batch's completion clock: every problem's records are complete
    before its objectives are written, both within the evaluation's own time
    (CUDA events around it), and problems of different sizes complete at
    different times; a graph replay stamps them again."""
    probs = _problems()
    gps = [mo.Problem(p) for p in probs]
    batch = mo.Batch(gps)
    srcs = [torch.as_tensor(p.sol_src).cuda() for p in probs]
    tgts = [torch.as_tensor(p.sol_tgt).cuda() for p in probs]
    outs = mo.Batch.outputs(srcs)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.eval_full(srcs, tgts, outs, stream=stream)
        batch.capture(srcs, tgts, outs, stream)
    stream.synchronize()
    for run in range(2):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            if run == 0:
                batch.eval_full(srcs, tgts, outs, stream=stream)
            else:
                batch.replay(stream)
            b.record(stream)
        b.synchronize()
        total = a.elapsed_time(b)
        rec, obj = batch.latency()
        assert (rec > 0).all() and (obj >= rec).all(), (rec, obj)
        assert obj.max() <= total * 1.05 + 0.05, (obj, total)
        assert len(np.unique(np.round(rec, 4))) > 1
