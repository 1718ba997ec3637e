"""Batched (grouped) factorizations of uneven N against single-instance runs and the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_2404_19163_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [100, 257, 64, 300, 129, 513, 1, 700]


@pytest.fixture(scope="module")
def ctx():
    from paper_2404_19163_gb300 import Context, build
    build.build()
    c = Context(0)
    yield c
    c.close()


def mats(sizes, seed=0):
    out = []
    for k, n in enumerate(sizes):
        if k % 2 == 0:
            S, Q, lam = synth.householder_spd(n, seed=seed * 100 + k)
        else:
            pos = synth.cluster_sites(n, seed * 100 + k)
            S = synth.gaussian_overlap(pos)
        out.append(S)
    return out


@pytest.mark.parametrize("prec", ["bf16", "bf16_split"])
def test_batched_matches_single_instance(ctx, prec):
    import torch
    Ss = mats(SIZES)
    St = [torch.from_numpy(S).cuda() for S in Ss]
    Zb, hist, infos, status = ctx.refine_batched(St, None, precision=prec, hist_cap=32)
    assert all(s in (0, 100) for s in status), status
    for k, S in enumerate(Ss):
        n = S.shape[0]
        # the single-instance path from the same start as a dense matrix: a cold start (Z0 = NULL)
        # would form its first residual and update elementwise, more accurately than the grouped
        # products, and the (h)(h) histories would then differ at the BF16 level
        Z0 = torch.eye(n, dtype=torch.float64, device="cuda") * oracle.gershgorin_scale(S)
        r = ctx.refine(St[k], Z0, order=2, precision=prec, refine_steps=0)
        # same arithmetic per instance: the same stop iteration and the same history
        assert infos[k]["iters"] == r.info["iters"], (k, infos[k], r.info)
        h = hist[k][:infos[k]["hist_len"]]
        assert np.allclose(h, r.hist[:len(h)], rtol=1e-3, atol=1e-6), (k, h, r.hist)
        Z = Zb[k].cpu().numpy()
        # the FP64-accurate final residual reported for instance k is the oracle's residual of Z_k
        _, e = oracle.residual(S, Z)
        assert abs(infos[k]["resid_f"] - e) <= 1e-12 + 1e-9 * e
        floor = 2.0 ** -7 if prec == "bf16" else 2.0 ** -14
        assert e / math.sqrt(n) <= floor


def test_batched_warm_start_frames(ctx):
    """Frame f+1 starts from frame f's Z (sites displaced by 0.02): it needs fewer updates."""
    import torch
    sizes = [300, 180, 420]
    base = [synth.cluster_sites(n, 900 + k) for k, n in enumerate(sizes)]
    g = np.random.default_rng(5)
    S0 = [torch.from_numpy(synth.gaussian_overlap(p)).cuda() for p in base]
    Z0, h0, i0, s0 = ctx.refine_batched(S0, None, precision="bf16_split")
    moved = [p + g.normal(0, 0.02, p.shape) for p in base]
    S1 = [torch.from_numpy(synth.gaussian_overlap(p)).cuda() for p in moved]
    Z1, h1, i1, s1 = ctx.refine_batched(S1, Z0, precision="bf16_split")
    for k in range(3):
        assert h1[k][0] < 0.1 * h0[k][0]          # the warm start is much closer
        assert i1[k]["iters"] <= i0[k]["iters"]
        _, e = oracle.residual(S1[k].cpu().numpy(), Z1[k].cpu().numpy())
        assert e / math.sqrt(sizes[k]) <= 2.0 ** -14


def test_batched_fixed_iters_and_errors(ctx):
    import torch
    from paper_2404_19163_gb300 import ZfactError
    Ss = [torch.from_numpy(S).cuda() for S in mats([90, 200], seed=3)]
    Zb, hist, infos, status = ctx.refine_batched(Ss, None, precision="bf16", fixed_iters=2)
    assert [i["iters"] for i in infos] == [2, 2]
    Sn = np.eye(50)
    Sn[3, 4] = Sn[4, 3] = np.nan
    with pytest.raises(ZfactError):
        ctx.refine_batched([Ss[0], torch.from_numpy(Sn).cuda()], None, precision="bf16")


def test_batched_residuals_of_mixed_conditioning(ctx):
    """Every instance gets the slice count of its own dynamic range (as the single-instance path
    does), so the reported residual of an ill-conditioned member (fcc block, cond ~7e4) agrees with
    the oracle's FP64 residual of the returned Z as closely as the well-conditioned members'."""
    import torch
    Ss = [synth.fcc_overlap(cells=(2, 2, 4)), synth.householder_spd(300, seed=5)[0],
          synth.gaussian_overlap(synth.cluster_sites(200, 7)), synth.fcc_overlap(cells=(2, 2, 2))]
    St = [torch.from_numpy(S).cuda() for S in Ss]
    Z, hist, info, status = ctx.refine_batched(St, None, precision="bf16_split")
    for S, z, inf in zip(Ss, Z, info):
        _, e = oracle.residual(S, z.cpu().numpy())
        assert abs(inf["resid_f"] - e) <= 1e-6 * e, (inf["resid_f"], e)


def test_batched_with_refinement_reaches_fp64(ctx):
    """refine_steps > 0: every instance gets Algorithm 3's sliced refinement after the grouped bulk and
    reaches 1e-12, checked with the oracle's residual of the returned Z."""
    import torch
    Ss = mats([100, 257, 300, 64])
    St = [torch.from_numpy(S).cuda() for S in Ss]
    Z, hist, info, status = ctx.refine_batched(St, None, precision="bf16_split", refine_steps=2, tol=1e-12)
    for S, z, h, inf in zip(Ss, Z, hist, info):
        n = S.shape[0]
        _, e = oracle.residual(S, z.cpu().numpy())
        assert inf["refine_iters"] >= 1 and inf["resid_f"] / math.sqrt(n) <= 1e-12
        assert e / math.sqrt(n) <= 1e-12 and abs(inf["resid_f"] - e) <= 1e-12
        assert inf["hist_len"] > inf["iters"] + 1


@pytest.mark.parametrize("emu", ["auto", "slices"])
def test_batched_final_residuals_grouped(ctx, emu):
    """Under the default scheme every instance's FP64-accurate final residual comes from grouped launches
    (two residue-product launches for the whole batch, which fits one group), and each equals the
    oracle's residual of the returned Z; with slices requested the per-instance lanes run instead."""
    import torch
    sizes = [300, 64, 513, 1, 129, 700, 257, 100, 450, 33]
    Ss = mats(sizes, seed=3)
    St = [torch.from_numpy(S).cuda() for S in Ss]
    ctx.set_emulation(emu)
    ctx.set_profiling(True)
    ctx.kernel_stats(reset=True)
    try:
        Zb, hist, infos, status = ctx.refine_batched(St, None, precision="bf16_split", hist_cap=32)
        stats = {k["name"]: k for k in ctx.kernel_stats(reset=True)}
    finally:
        ctx.set_profiling(False)
        ctx.set_emulation("auto")
    assert all(s in (0, 100) for s in status), status
    if emu == "auto":
        assert stats["tc_gemm.crt"]["launches"] == 2, stats.get("tc_gemm.crt")
    else:
        assert "tc_gemm.crt" not in stats and stats["tc_gemm.ozaki"]["launches"] >= len(sizes)
    for k, S in enumerate(Ss):
        _, e = oracle.residual(S, Zb[k].cpu().numpy())
        assert abs(infos[k]["resid_f"] - e) <= 1e-12 + 1e-9 * e, (k, infos[k]["resid_f"], e)
