"""The benchmark's own configuration against the FP64 oracle.

bench.py times one factorization of the N = 4096 cubic Gaussian overlap: cold start
Z0 = I / sqrt(g_hi), m = 2, the BF16 hi/lo split bulk (Sec. 3.2, Eqs. SZn, Xn, Xsq),
then Algorithm 3's refinement with d and Z + Z Q formed to FP64 accuracy by the default
product scheme (CRT residues), to ||I - Z^T S Z||_F / sqrt(N) <= 1e-12.  Here the same
call's Z is checked with the oracle's FP64 residual, and the library's FP64-accurate d of
that Z is compared with the oracle's d element by element.

Tolerance of the element-wise comparison: both d are FP64-accurate evaluations of the same
I - Z^T S Z, so they differ by rounding on the scale of |Z|^T |S| |Z| (FP64 products) and
the 2^-54 row-scaled fixed point of the residue operands: 1e-13 max(|Z|^T |S| |Z|) holds
with two orders to spare.  Their Frobenius norms then differ by at most N times that."""
import math

import numpy as np
import pytest

import oracle
from paper_2404_19163_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    from paper_2404_19163_gb300 import Context, build
    build.build()
    c = Context(0)
    yield c
    c.close()


def _headline_run(ctx, S):
    import torch
    St = torch.from_numpy(S).cuda()
    r = ctx.refine(St, None, order=2, precision="bf16_split", tol=TOL)
    return St, r


def _check(ctx, S, St, r):
    import torch
    n = S.shape[0]
    Z = r.Z.cpu().numpy()
    d_or, err_or = oracle.residual(S, Z)
    assert err_or / math.sqrt(n) <= TOL, err_or / math.sqrt(n)
    assert r.info["resid_f"] / math.sqrt(n) <= TOL
    scale = float(np.max(np.abs(Z).T @ (np.abs(S) @ np.abs(Z))))
    assert abs(r.info["resid_f"] - err_or) <= 1e-13 * scale * n, (r.info["resid_f"], err_or)
    D = torch.empty_like(St)
    err = ctx.residual(St, r.Z, "ozaki", D=D)
    assert err == r.info["resid_f"] or abs(err - r.info["resid_f"]) <= 1e-13 * scale * n
    diff = np.abs(D.cpu().numpy() - d_or)
    assert float(np.max(diff)) <= 1e-13 * scale, float(np.max(diff)) / scale
    return Z, err_or


def test_headline_configuration_n1500_elementwise(ctx):
    """The same configuration on a 1500-site block of the workload's lattice (three 512-wide K
    ranges and a ragged tail of 236): the full d element by element."""
    S = synth.cubic_overlap(n_side=12)[:1500, :1500].copy()
    St, r = _headline_run(ctx, S)
    assert r.info["refine_iters"] >= 1
    _check(ctx, S, St, r)


def test_headline_configuration_n4096(ctx):
    """The benchmark's workload itself (N = 4096), the oracle's FP64 residual of the returned Z."""
    S = synth.cubic_overlap()
    assert S.shape == (4096, 4096)
    ctx.set_profiling(True)
    ctx.kernel_stats(reset=True)
    St, r = _headline_run(ctx, S)
    names = {k["name"] for k in ctx.kernel_stats()}
    ctx.set_profiling(False)
    assert "tc_gemm.crt" in names, names        # the refinement ran on CRT residues
    Z, err_or = _check(ctx, S, St, r)
    # the FP64 GPU path's factor is another valid factor; the two agree to the bulk's accuracy
    assert r.info["iters"] >= 2 and r.info["refine_iters"] >= 1


@pytest.mark.parametrize("refine_steps", [3, 0])
def test_pinned_host_output_is_the_device_result(ctx, refine_steps):
    """A pinned host Z (the end-to-end path) receives the result by a copy started after the last
    refinement update, overlapping the final residual; it must hold exactly the device result, also
    when no update follows the copy's source (bulk only) and when S comes from the host too."""
    import torch
    S = synth.cubic_overlap(n_side=10)
    n = S.shape[0]
    St = torch.from_numpy(S).cuda()
    kw = dict(order=2, precision="bf16_split", tol=TOL if refine_steps else 0.0, refine_steps=refine_steps)
    rd = ctx.refine(St, None, **kw)
    Zh = torch.empty((n, n), dtype=torch.float64).pin_memory()
    Sh = torch.from_numpy(S).pin_memory()
    rh = ctx.refine(Sh, None, Z=Zh, **kw)
    assert torch.equal(Zh, rd.Z.cpu())
    assert rh.info["iters"] == rd.info["iters"] and rh.info["refine_iters"] == rd.info["refine_iters"]
    assert rh.info["resid_f"] == rd.info["resid_f"] or (math.isnan(rh.info["resid_f"]) and math.isnan(rd.info["resid_f"]))
    # a pageable host Z takes the copy at the end
    Zp = np.empty((n, n))
    ctx.refine(St, None, Z=Zp, **kw)
    assert np.array_equal(Zp, rd.Z.cpu().numpy())
