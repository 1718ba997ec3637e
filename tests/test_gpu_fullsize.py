"""Full-size workloads in the launch configuration bench.py times, checked through properties
that hold at any size, residual columns formed in about twice FP64 precision, and host recomputations."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2404_19163_gb300 import Context, build
    build.build()
    c = Context(0)
    yield c
    c.close()


def test_workload3_ill_conditioned_warm_start(ctx):
    """N = 16384 fcc overlap (cond ~7.5e5), Z0 from the displaced geometry, FP16 hi/lo bulk and
    sliced FP64-accurate refinement to 1e-12.  Sampled columns of d, formed in about twice FP64
    precision, show the sliced residual to be at least as accurate as FP64 arithmetic."""
    import torch
    from paper_2404_19163_gb300 import synth
    import accurate_dot as ad
    S = synth.fcc_overlap_torch()
    n = S.shape[0]
    Sp = synth.fcc_overlap_torch(perturb=0.01)
    Z0 = ctx.refine(Sp, None, order=2, precision="fp16_split", tol=0.0).Z
    del Sp
    r = ctx.refine(S, Z0, order=2, precision="fp16_split", tol=1e-12)
    assert r.info["resid_f"] / math.sqrt(n) <= 1e-12
    D = torch.empty_like(S)
    Dn = torch.empty_like(S)
    e_oz = ctx.residual(S, r.Z, "ozaki", D=D)
    e_native = ctx.residual(S, r.Z, "native", D=Dn)
    assert abs(e_oz - r.info["resid_f"]) <= 1e-3 * r.info["resid_f"]
    # native FP64 adds its own rounding noise to d, so it can only read a larger norm
    assert r.info["resid_f"] <= 1.05 * e_native
    for j in (0, 7777, n - 1):
        ref = ad.residual_column(S, r.Z, j)
        err_oz = float(torch.linalg.norm(D[:, j] - ref))
        err_native = float(torch.linalg.norm(Dn[:, j] - ref))
        assert err_oz <= err_native, (j, err_oz, err_native, float(torch.linalg.norm(ref)))


def test_workload4_batched_frame(ctx):
    """The batched trajectory at full size for one warm frame: every instance ends at the split-BF16
    bulk floor and its reported FP64-accurate residual is the one the host computes for a sample."""
    import torch
    from paper_2404_19163_gb300 import synth
    sizes, frame = synth.trajectory(count=128)
    S0 = [synth.gaussian_overlap_torch(p) for p in frame.positions(0)]
    Z0, h0, i0, s0 = ctx.refine_batched(S0, None, precision="bf16_split")
    del S0
    S1 = [synth.gaussian_overlap_torch(p) for p in frame.positions(1)]
    Z1, h1, i1, s1 = ctx.refine_batched(S1, Z0, precision="bf16_split")
    assert all(s in (0, 100) for s in s1)
    res = np.array([i["resid_f"] / math.sqrt(n) for i, n in zip(i1, sizes)])
    assert np.all(res <= 2.0 ** -14)
    assert np.mean([i["iters"] for i in i1]) < np.mean([i["iters"] for i in i0])
    k = int(np.argmin(sizes))
    Sh = S1[k].cpu().numpy()
    Zh = Z1[k].cpu().numpy()
    d = np.eye(Sh.shape[0]) - Zh.T @ Sh @ Zh
    assert abs(np.linalg.norm(d) - i1[k]["resid_f"]) <= 1e-10 * max(1.0, i1[k]["resid_f"])
