"""tcgen05 tensor-core products and the mixed-precision recursion against the oracle.

Step-level parity: the GPU product of 16-bit operands (FP32 accumulation in
tensor memory) is compared element by element with the oracle's FP64 product
of the same 16-bit-rounded operands.  The difference is FP32 accumulation
rounding only, bounded by (nseg*K) * 2^-23 * (|A16| |B16|)_ij (any summation
order, truncating or rounding adder)."""
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


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


KIND = {"bf16": "bf16", "bf16_split": "bf16", "fp16": "fp16", "fp16_split": "fp16"}


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_split_bit_exact(ctx, prec):
    import torch
    g = np.random.default_rng(1)
    A = g.standard_normal(100003) * 10.0 ** g.uniform(-3, 3, 100003)
    scale = 2.0 ** -3 if prec == "fp16" else 1.0
    hi, lo = ctx.split(dev(A), prec, scale)
    rh, rl = oracle.split16(A, KIND[prec], scale)
    np16 = np.float16 if prec == "fp16" else None
    if prec == "fp16":
        eh = rh.astype(np.float16).view(np.uint16)
        el = rl.astype(np.float16).view(np.uint16)
    else:
        eh = (rh.view(np.uint32) >> 16).astype(np.uint16)
        el = (rl.view(np.uint32) >> 16).astype(np.uint16)
    assert np.array_equal(hi.cpu().numpy().view(np.uint16), eh)
    assert np.array_equal(lo.cpu().numpy().view(np.uint16), el)


@pytest.mark.parametrize("n", [128, 64, 129, 256, 300, 520])
@pytest.mark.parametrize("prec", ["bf16", "fp16", "bf16_split", "fp16_split"])
def test_gemm_parity(ctx, n, prec):
    g = np.random.default_rng(n)
    A = g.standard_normal((n, n))
    B = g.standard_normal((n, n)) * 0.5
    sa, sb = (2.0 ** 4, 2.0 ** -2) if prec.startswith("fp16") else (1.0, 1.0)
    C = ctx.gemm(dev(A), dev(B), prec, sa, sb).cpu().numpy()
    kind = KIND[prec]
    Ah, Al = oracle.split16(A, kind, sa)
    Bh, Bl = oracle.split16(B, kind, sb)
    if prec.endswith("split"):
        ref = oracle.mm16(Ah, Bh) + oracle.mm16(Ah, Bl) + oracle.mm16(Al, Bh)
        absp = np.abs(Ah) @ np.abs(Bh) + np.abs(Ah) @ np.abs(Bl) + np.abs(Al) @ np.abs(Bh)
        nseg = 3
    else:
        ref = oracle.mm16(Ah, Bh)
        absp = np.abs(Ah) @ np.abs(Bh)
        nseg = 1
    ref /= sa * sb
    bound = nseg * n * 2.0 ** -23 * absp / (sa * sb) + 1e-30
    err = np.abs(C - ref)
    assert np.all(err <= bound), (prec, n, float(np.max(err / bound)))
    # the exact FP64 product differs by the operand rounding only
    full = A @ B
    u = 2.0 ** -8 if kind == "bf16" else 2.0 ** -11
    if prec.endswith("split"):
        u = u * u * 4
    assert np.max(np.abs(C - full)) <= 4 * u * np.max(np.abs(A) @ np.abs(B)) + 1e-6


def test_mixed_bf16_workload1(ctx):
    S, Q, lam = synth.householder_spd(256, seed=0)
    n = 256
    Zo, ho, it = oracle.refine(S, None, m=2, nmax=50)
    r = ctx.refine(dev(S), None, order=2, precision="bf16", tol=1e-12)
    Z = r.Z.cpu().numpy()
    res = np.linalg.norm(np.eye(n) - Z.T @ S @ Z) / math.sqrt(n)
    assert res <= 1e-12
    assert r.info["resid_f"] / math.sqrt(n) <= 1e-12
    # a different but valid factor: Z = S^{-1/2} U, U orthogonal within the BF16 floor
    relz = np.linalg.norm(Z - Zo) / np.linalg.norm(Zo)
    assert relz <= 5e-2
    assert r.info["launches"] > 0
    assert np.linalg.norm(Z @ Z.T - np.linalg.inv(S)) / np.linalg.norm(np.linalg.inv(S)) <= 1e-11


@pytest.mark.parametrize("prec", ["bf16", "bf16_split", "fp16", "fp16_split", "fp32"])
def test_mixed_bulk_history_tracks_fp64(ctx, prec):
    """Before the BF16 noise floor, Err_n of the mixed bulk follows the FP64 oracle's."""
    S = synth.cubic_overlap(n_side=8)
    n = S.shape[0]
    Zo, ho, it = oracle.refine(S, None, m=2, nmax=50, fixed_iters=2)
    r = ctx.refine(dev(S), None, order=2, precision=prec, fixed_iters=2, refine_steps=0)
    u = {"bf16": 2.0 ** -8, "bf16_split": 2.0 ** -16, "fp16": 2.0 ** -11, "fp16_split": 2.0 ** -20,
         "fp32": 2.0 ** -22}[prec]
    for k in range(3):
        assert abs(r.hist[k] - ho[k]) <= 8 * u * math.sqrt(n) + 1e-3 * ho[k], (k, r.hist, ho)


@pytest.mark.parametrize("m", [3, 4])
def test_mixed_higher_order(ctx, m):
    S, Q, lam = synth.householder_spd(200, seed=m)
    r = ctx.refine(dev(S), None, order=m, precision="bf16", tol=1e-12)
    assert r.info["resid_f"] / math.sqrt(200) <= 1e-12


@pytest.mark.parametrize("n,prec", [(1, "bf16_split"), (7, "fp16_split"), (100, "bf16_split"), (129, "fp16"),
                                    (383, "fp16_split"), (150, "fp32")])
def test_mixed_ragged(ctx, n, prec):
    S, Q, lam = synth.householder_spd(n, seed=n)
    r = ctx.refine(dev(S), None, order=2, precision=prec, tol=1e-12, refine_steps=3)
    Z = r.Z.cpu().numpy()
    assert np.linalg.norm(np.eye(n) - Z.T @ S @ Z) / math.sqrt(n) <= 1e-12


def test_mixed_workload2_full_size(ctx):
    """N = 4096 Gaussian overlap, BF16 bulk + FP64-d refinement, to tol 1e-12."""
    S = synth.cubic_overlap()
    n = S.shape[0]
    r = ctx.refine(dev(S), None, order=2, precision="bf16", tol=1e-12)
    assert r.info["resid_f"] / math.sqrt(n) <= 1e-12
    # sampled entries of d = I - Z^T S Z, each recomputed by the oracle's definition in FP64
    Z = r.Z.cpu().numpy()
    g = np.random.default_rng(3)
    A_cols = {}
    for _ in range(16):
        i, j = g.integers(0, n, 2)
        sz_j = S @ Z[:, j]
        d_ij = (1.0 if i == j else 0.0) - float(np.dot(Z[:, i], sz_j))
        assert abs(d_ij) <= 1e-12 * 10


@pytest.mark.parametrize("prec", ["fp16", "fp16_split"])
def test_mixed_fp16_scaled_operands(ctx, prec):
    """FP16 operands carry power-of-two scales: a badly scaled S (entries ~1e-3, so FP16
    without scaling would lose the lo parts to subnormals) still converges to tol."""
    S, Q, lam = synth.householder_spd(160, seed=21)
    S = S * 1e-3
    r = ctx.refine(dev(S), None, order=2, precision=prec, tol=1e-12)
    Z = r.Z.cpu().numpy()
    _, e = oracle.residual(S, Z)
    assert e / math.sqrt(160) <= 1e-12
    assert r.info["iters"] >= 1


def test_fp16_split_bulk_floor_below_bf16(ctx):
    """The split scheme's bulk floor (Sec. 3.2) sits far below plain BF16's."""
    S = synth.cubic_overlap(n_side=10)
    r1 = ctx.refine(dev(S), None, order=2, precision="bf16", refine_steps=0)
    r2 = ctx.refine(dev(S), None, order=2, precision="fp16_split", refine_steps=0)
    b1 = min(r1.hist[:r1.info["iters"] + 1])
    b2 = min(r2.hist[:r2.info["iters"] + 1])
    assert b2 < 1e-2 * b1, (r1.hist, r2.hist)


@pytest.mark.parametrize("n", [64, 129, 300, 2049])
def test_fp32_gemm_parity(ctx, n):
    """The paper's "single" product: FP32 operands, FP32 CUDA-core accumulation."""
    g = np.random.default_rng(40 + n)
    A = g.standard_normal((n, n))
    B = g.standard_normal((n, n))
    C = ctx.gemm(dev(A), dev(B), "fp32").cpu().numpy()
    A32 = A.astype(np.float32).astype(np.float64)
    B32 = B.astype(np.float32).astype(np.float64)
    ref = A32 @ B32
    bound = n * 2.0 ** -23 * (np.abs(A32) @ np.abs(B32))
    assert np.all(np.abs(C - ref) <= bound)


def test_fp32_single_path_reaches_its_floor_and_refines(ctx):
    S, Q, lam = synth.householder_spd(200, seed=31)
    r = ctx.refine(dev(S), None, order=2, precision="fp32")
    _, e = oracle.residual(S, r.Z.cpu().numpy())
    assert e / math.sqrt(200) <= 1e-5 and abs(r.info["resid_f"] - e) <= 1e-12
    r2 = ctx.refine(dev(S), None, order=2, precision="fp32", refine_steps=2, tol=1e-12)
    _, e2 = oracle.residual(S, r2.Z.cpu().numpy())
    assert e2 / math.sqrt(200) <= 1e-12


def test_hh_with_single_precision_refinement(ctx):
    """Table I's "(h)(h)+refi" with its FP32 step: from the BF16 (h)(h) bulk, one refinement update
    with d, Q and Z + ZQ in FP32 takes the residual far below the bulk's floor but not to FP64's;
    the history holds the step's FP32 Err and then the FP64-accurate residual of the returned Z."""
    S = synth.cubic_overlap(n_side=10)
    n = S.shape[0]
    rb = ctx.refine(dev(S), None, order=2, precision="bf16", refine_steps=0)
    r = ctx.refine(dev(S), None, order=2, precision="bf16", refine_mode="fp32", refine_steps=1)
    assert r.info["iters"] == rb.info["iters"] and r.info["refine_iters"] == 1
    assert len(r.hist) == r.info["iters"] + 3 and r.hist[-1] == r.info["resid_f"]
    _, e = oracle.residual(S, r.Z.cpu().numpy())
    assert abs(r.info["resid_f"] - e) <= 1e-3 * e
    assert e < 1e-2 * rb.info["resid_f"]
    assert 1e-10 <= e / math.sqrt(n) <= 1e-5


def test_unknown_refine_mode_rejected(ctx):
    from paper_2404_19163_gb300.zfact import ZfactError
    S, Q, lam = synth.householder_spd(64, seed=2)
    with pytest.raises(ZfactError) as ei:
        ctx.refine(dev(S), None, order=2, precision="bf16", refine_mode=7)
    assert ei.value.code == 1


@pytest.mark.parametrize("n", [64, 129, 256, 520])
def test_gemm_fp16_accumulator(ctx, n):
    """Table I's (h)(h)half: FP16 operands and an FP16 accumulator.  Against the oracle's FP64
    product of the same FP16 operands the error is the accumulator's rounding: at most one FP16
    rounding (relative 2^-11, absolute 2^-25 below FP16's normal range) of a partial sum bounded by
    (|A16| |B16|)_ij after each K = 16 step and once at the end.  The FP32-accumulating product of
    the same operands is far more accurate, which shows the accumulator really is FP16."""
    g = np.random.default_rng(100 + n)
    A = g.standard_normal((n, n))
    B = g.standard_normal((n, n)) * 0.5
    sa, sb = 2.0 ** -3, 2.0 ** -2   # scaled operands at most about 1
    C = ctx.gemm(dev(A), dev(B), "fp16_half", sa, sb).cpu().numpy()
    C32 = ctx.gemm(dev(A), dev(B), "fp16", sa, sb).cpu().numpy()
    Ah, _ = oracle.split16(A, "fp16", sa)
    Bh, _ = oracle.split16(B, "fp16", sb)
    ref = oracle.mm16(Ah, Bh)
    absp = np.abs(Ah).astype(np.float64) @ np.abs(Bh).astype(np.float64)
    steps = -(-n // 16) + 2
    bound = steps * (2.0 ** -11 * absp + 2.0 ** -25)
    err = np.abs(C * (sa * sb) - ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    err32 = np.abs(C32 * (sa * sb) - ref)
    assert np.max(err) > 30 * np.max(err32), (float(np.max(err)), float(np.max(err32)))


def test_fp16_half_bulk_contracts_and_refines(ctx):
    """(h)(h)half bulk: Algorithm 2 contracts Err from the cold start and stops at a floor above
    the FP32-accumulating (h)(h)'s; Algorithm 3's FP64-accurate refinement then reaches 1e-12."""
    S = synth.cubic_overlap(n_side=8)
    n = S.shape[0]
    rh = ctx.refine(dev(S), None, order=2, precision="fp16_half", refine_steps=0)
    r16 = ctx.refine(dev(S), None, order=2, precision="fp16", refine_steps=0)
    bh = min(rh.hist[:rh.info["iters"] + 1])
    b16 = min(r16.hist[:r16.info["iters"] + 1])
    assert rh.info["iters"] >= 2 and bh < 1e-2 * rh.hist[0], rh.hist
    assert bh > b16, (rh.hist, r16.hist)
    r = ctx.refine(dev(S), None, order=2, precision="fp16_half", tol=1e-12, refine_steps=4)
    _, e = oracle.residual(S, r.Z.cpu().numpy())
    assert e / math.sqrt(n) <= 1e-12
