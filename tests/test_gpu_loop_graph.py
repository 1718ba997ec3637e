"""The device-driven bulk loop (zfact_set_loop_graphs): Algorithm 2's updates after the first run as
one CUDA graph whose while node applies the stop test on the device.  It launches the same kernels
with the same arguments as the host-driven loop, so the two must agree bit for bit: the returned Z,
the Err history, the update count."""
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
    c.set_loop_graphs(True)
    c.close()


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(ctx, S, graphs, **kw):
    ctx.set_loop_graphs(graphs)
    ctx.set_profiling(True)
    ctx.kernel_stats(reset=True)
    r = ctx.refine(S, None, **kw)
    names = {k["name"] for k in ctx.kernel_stats(reset=True)}
    ctx.set_profiling(False)
    return r, names


@pytest.mark.parametrize("precision,order", [("bf16_split", 2), ("fp16_split", 3), ("bf16", 2)])
@pytest.mark.parametrize("n", [300, 1100])
def test_graph_loop_matches_host_loop(ctx, precision, order, n):
    S, Q, lam = synth.householder_spd(n, seed=20 + n)
    Sd = dev(S)
    kw = dict(order=order, precision=precision, refine_steps=0, final_residual=0)
    rh, nh = run(ctx, Sd, False, **kw)
    rg, ng = run(ctx, Sd, True, **kw)
    assert rh.info["iters"] >= 2          # so that the graph ran at least one update
    assert "bulk_graph" in ng and "bulk_graph" not in nh
    assert rg.info["iters"] == rh.info["iters"]
    assert np.array_equal(rg.hist, rh.hist)
    assert np.array_equal(rg.Z.cpu().numpy(), rh.Z.cpu().numpy())


def test_graph_loop_full_path_and_limit(ctx):
    """The full path (refinement after the graph-driven bulk) meets tol, checked with the oracle's
    residual; with nmax = 3 the graph stops at the third update although the stop test has not fired."""
    S = synth.cubic_overlap(n_side=11)
    n = S.shape[0]
    Sd = dev(S)
    r, names = run(ctx, Sd, True, order=2, precision="bf16_split", tol=1e-12)
    assert "bulk_graph" in names
    _, err = oracle.residual(S, r.Z.cpu().numpy())
    assert err / math.sqrt(n) <= 1e-12
    Sh, _, _ = synth.householder_spd(400, seed=3)    # cond 25: about 7 updates to the stop
    rl, _ = run(ctx, dev(Sh), True, order=2, precision="bf16_split", refine_steps=0, final_residual=0, nmax=3)
    rh, _ = run(ctx, dev(Sh), False, order=2, precision="bf16_split", refine_steps=0, final_residual=0, nmax=3)
    assert rl.info["iters"] == 3 == rh.info["iters"]
    assert np.array_equal(rl.Z.cpu().numpy(), rh.Z.cpu().numpy())
