"""Learned start proposal: the library's feature, MLP forward/backward and Adam kernels
against the FP64 CPU oracle, the proposal's fallback, and what a trained network gains
over the plain schedule (Gershgorin scale, m = 2)."""
import math

import numpy as np
import pytest

import oracle
from paper_2404_19163_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2404_19163_gb300 import Context, build
    build.build()
    c = Context(0)
    yield c
    c.close()


def dev(a, dt=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t if dt is None else t.to(dt)


@pytest.mark.parametrize("kind", ["householder", "cubic", "fcc"])
def test_features_match_oracle(ctx, kind):
    if kind == "householder":
        S, _, _ = synth.householder_spd(200, seed=4)
    elif kind == "cubic":
        S = synth.cubic_overlap(n_side=7)
    else:
        S = synth.fcc_overlap(cells=(2, 2, 3), a_lat=3.6)
    f = ctx.features(dev(S))
    fo = oracle.features(S)
    scale = np.maximum(np.abs(fo), 1e-3)
    assert np.all(np.abs(f - fo) <= 2e-4 * scale + 1e-6), np.max(np.abs(f - fo) / scale)


def random_net(seed):
    g = np.random.default_rng(seed)
    P = (g.standard_normal(oracle.mlp_num_params()) * 0.3)
    x = g.standard_normal((37, 16)) * 2.0 + 1.0
    mean = x.mean(axis=0)
    std = x.std(axis=0) + 0.1
    return P, x, mean, std


def test_mlp_forward_matches_oracle(ctx):
    import torch
    P, x, mean, std = random_net(1)
    y = ctx.mlp_forward(dev(P, torch.float32), dev(mean, torch.float32), dev(std, torch.float32),
                        dev(x, torch.float32)).cpu().numpy()
    xn = ((x.astype(np.float32) - mean.astype(np.float32)) / std.astype(np.float32)).astype(np.float64)
    yo = oracle.mlp_forward(P.astype(np.float32).astype(np.float64), xn)
    assert np.allclose(y, yo, rtol=1e-4, atol=1e-4)


def test_mlp_backward_matches_oracle(ctx):
    import torch
    P, x, mean, std = random_net(2)
    g = np.random.default_rng(3)
    ts = g.standard_normal(37).astype(np.float32)
    to = g.integers(0, 4, 37).astype(np.int32)
    grad, loss = ctx.mlp_backward(dev(P, torch.float32), dev(mean, torch.float32), dev(std, torch.float32),
                                  dev(x, torch.float32), dev(ts), dev(to), 0.7)
    xn = ((x.astype(np.float32) - mean.astype(np.float32)) / std.astype(np.float32)).astype(np.float64)
    P64 = P.astype(np.float32).astype(np.float64)
    go = oracle.mlp_backward(P64, xn, ts.astype(np.float64), to, 0.7)
    lo = oracle.mlp_loss(P64, xn, ts.astype(np.float64), to, 0.7)
    gg = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - go) <= 1e-4 * np.linalg.norm(go)
    assert abs(loss - lo) <= 1e-5 * abs(lo)


def test_adam_matches_oracle(ctx):
    import torch
    g = np.random.default_rng(4)
    p = g.standard_normal(1000).astype(np.float32)
    gr = g.standard_normal(1000).astype(np.float32)
    m = (g.standard_normal(1000) * 0.1).astype(np.float32)
    v = (g.random(1000) * 0.1).astype(np.float32)
    P, G, M, V = dev(p), dev(gr), dev(m), dev(v)
    ctx.mlp_adam(P, G, M, V, 7, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8)
    # the kernel receives its hyper-parameters as FP32: give the oracle the same values
    f32 = lambda x: float(np.float32(x))
    po, mo, vo = oracle.adam_step(p.astype(np.float64), gr.astype(np.float64), m.astype(np.float64),
                                  v.astype(np.float64), 7, lr=f32(1e-2), b1=f32(0.9), b2=f32(0.999), eps=f32(1e-8))
    assert np.allclose(P.cpu().numpy(), po, rtol=1e-5, atol=1e-6)
    assert np.allclose(M.cpu().numpy(), mo, rtol=1e-5, atol=1e-7)
    assert np.allclose(V.cpu().numpy(), vo, rtol=1e-5, atol=1e-9)


def test_propose_fallback_and_decoding(ctx):
    import torch
    S, _, _ = synth.householder_spd(150, seed=6)
    s0 = oracle.gershgorin_scale(S)
    P = np.zeros(oracle.mlp_num_params(), dtype=np.float32)
    mean = dev(np.zeros(16, np.float32))
    std = dev(np.ones(16, np.float32))
    # b3 = (log 1.3, logits favouring m = 4)
    P[-5:] = [math.log(1.3), 0.0, 0.1, 2.0, 0.5]
    s, m = ctx.propose(dev(S), dev(P), mean, std)
    assert abs(s / s0 - 1.3) < 1e-5 and m == 4
    # an out-of-range scale falls back to the plain schedule
    P[-5] = 10.0
    s, m = ctx.propose(dev(S), dev(P), mean, std)
    assert abs(s / s0 - 1.0) < 1e-12 and m == 2


def test_training_pipeline_on_method_labels(ctx):
    """Labels from the method itself (grouped runs over the (f, m) grid), then training on the
    library's kernels: the loss falls by half, and the labels are the grid's modelled optimum."""
    from paper_2404_19163_gb300 import learn
    Str = learn.instances(160, "train", 128, 384)
    Xtr = learn.features(ctx, Str)
    ys, yo, table = learn.label(ctx, Str, Xtr)
    P, mu, sd, losses = learn.train(ctx, Xtr, ys, yo, steps=1500)
    assert losses[-1] < 0.5 * losses[0]
    flat = table.reshape(len(Str), -1)
    ok = np.isfinite(flat).any(axis=1)
    assert ok.mean() >= 0.75
    best = np.argmin(flat[ok], axis=1)
    fi, mi = np.unravel_index(best, table.shape[1:])
    assert np.allclose(ys[ok], np.log(np.asarray(learn.F_GRID))[fi]) and np.array_equal(yo[ok], mi)


def test_shipped_network_measured_gain(ctx):
    """The shipped network (trained on 20 000 method-labelled matrices, N in [128, 4096]) against the
    plain schedule (Gershgorin scale, m = 2) on held-out matrices of the same family, measured: device
    time of the whole path to tol (bulk, refinement, FP64-accurate final residual) and of the bulk.
    The proposal must converge wherever the plain schedule does (a start that does not contract falls
    back inside the call), take fewer bulk iterations, and cost no more than the plain schedule beyond
    timing noise."""
    from paper_2404_19163_gb300 import learn
    P, mu, sd, meta = learn.load()
    assert meta["train"] >= 20000 and meta["n_range"] == [128, 4096]
    ks = [k for k in range(400) if synth.proposal_sites(k, 128, 4096, "heldout")[0].shape[0] <= 1536][:40]
    rows = []
    for k in ks:
        rows += learn.evaluate(ctx, learn.instances(1, "heldout", 128, 4096, start=k), P, mu, sd)
    summ = learn.summarize(rows)
    print("measured on %d held-out matrices: full time %.1f -> %.1f ms (gain %.1f%%), bulk %.1f -> %.1f ms, "
          "bulk iterations %.2f -> %.2f" % (len(rows), summ["plain_ms"], summ["proposed_ms"],
                                            100 * summ["full_time_gain"], summ["plain_bulk_ms"],
                                            summ["proposed_bulk_ms"], summ["plain_iters"], summ["proposed_iters"]))
    assert all(r["prop_ok"] for r in rows if r["plain_ok"])
    assert summ["proposed_iters"] < summ["plain_iters"]
    assert summ["proposed_ms"] <= 1.03 * summ["plain_ms"]
