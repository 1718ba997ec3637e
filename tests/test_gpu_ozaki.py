"""FP64-accurate residual d = I - Z^T S Z by error-free slicing on the BF16 tensor
cores, against the FP64 oracle.  Row-scaled slicing is accurate normwise: the
truncation error of an entry is bounded by 2^-54 K times the row maxima of the
two factors, not by the entry's own |A||B|.  The bound used here,
1e-13 * max(|Z|^T |S| |Z|), is six orders below what plain FP32 accumulation
leaves (~1e-7), so it holds only if every slice-pair group is accumulated
exactly and combined in FP64."""
import math

import numpy as np
import pytest

import oracle
from paper_2404_19163_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["auto", "slices"])
def ctx(request):
    """Every test runs under both FP64-accurate product schemes: CRT residues where they fit
    (the default) and error-free slices."""
    from paper_2404_19163_gb300 import Context, build
    build.build()
    c = Context(0)
    c.set_emulation(request.param)
    c.emu = request.param
    yield c
    c.close()


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n", [5, 64, 200, 777, 1500, 3001, 4097, 4300])
def test_ozaki_residual_matches_oracle(ctx, n):
    import torch
    g = np.random.default_rng(n)
    if n <= 800:
        S, Q, lam = synth.householder_spd(n, seed=n)
        Z = (Q * lam ** -0.5) @ Q.T + 1e-3 * g.standard_normal((n, n))
    else:
        side = round(n ** (1 / 3)) + 1
        S = synth.cubic_overlap(n_side=side)[:n, :n].copy()
        Z = np.eye(n) / math.sqrt(np.abs(S).sum(axis=1).max()) + 1e-3 * g.standard_normal((n, n))
    d_or, err_or = oracle.residual(S, Z)
    D = torch.empty((n, n), dtype=torch.float64, device="cuda")
    err = ctx.residual(dev(S), dev(Z), "ozaki", D=D)
    scale = np.max(np.abs(Z).T @ np.abs(S) @ np.abs(Z))
    diff = np.abs(D.cpu().numpy() - d_or)
    assert np.max(diff) <= 1e-13 * scale, float(np.max(diff) / scale)
    assert abs(err - err_or) <= 1e-13 * scale * n
    # and the FP64 CUDA-core residual agrees too
    D2 = torch.empty_like(D)
    err2 = ctx.residual(dev(S), dev(Z), "native", D=D2)
    assert np.max(np.abs(D2.cpu().numpy() - d_or)) <= 1e-13 * scale


@pytest.mark.parametrize("n,zbits,sbits", [(300, 10, 4), (1500, 10, 4), (2048, 12, 3), (1201, 3, 3)])
def test_ozaki_residual_exact_on_integer_inputs(ctx, n, zbits, sbits):
    """Integer Z and S with X = Z^T S Z below 2^53: every partial sum is an integer FP64 holds, so
    the exact d = I - X is known and the sliced residual must reproduce it bit for bit (several
    K-chunks at n = 1500; more than 62 fixed-point bits at n = 2048)."""
    import torch
    g = np.random.default_rng(n + zbits)
    Z = g.integers(-2 ** zbits, 2 ** zbits, (n, n)).astype(np.float64)
    A = g.integers(-2 ** sbits, 2 ** sbits, (n, n)).astype(np.float64)
    S = A + A.T
    X = Z.T @ (S @ Z)
    assert np.abs(X).max() < 2.0 ** 52 and np.abs(S @ Z).max() < 2.0 ** 52
    D = torch.empty((n, n), dtype=torch.float64, device="cuda")
    ctx.residual(dev(S), dev(Z), "ozaki", D=D)
    assert np.array_equal(D.cpu().numpy(), np.eye(n) - X)


@pytest.mark.parametrize("n", [300, 4300, 8192])
def test_residual_exact_on_scaled_integer_inputs(ctx, n):
    """Integer Z scaled by 2^-20 and integer S, so max|Z|^2 times S's largest row sum is below one
    and the residual keeps 54 bits per operand: CRT residues under the default scheme (up to sixteen
    moduli; at N = 4300 and 8192 each residue product is summed in K-chunks of 1024 reduced modulo m
    in the epilogue).  Every product is an integer times a power of two that FP64 holds, so d
    must equal I - Z^T S Z bit for bit (columns sampled above N = 300)."""
    import torch
    g = np.random.default_rng(n)
    Zi = g.integers(-2 ** 8, 2 ** 8, (n, n)).astype(np.float64)
    A = g.integers(-8, 8, (n, n)).astype(np.float64)
    S = A + A.T
    cols = np.arange(n) if n <= 300 else np.unique(np.concatenate([g.choice(n, 24, replace=False), [0, n - 1]]))
    X = (Zi.T @ (S @ Zi[:, cols])) * 2.0 ** -40   # exact: integers below 2^47, then a power of two
    assert np.abs(Zi.T @ (S @ Zi[:, cols[:1]])).max() < 2.0 ** 52
    D = torch.empty((n, n), dtype=torch.float64, device="cuda")
    ctx.set_profiling(True)
    ctx.kernel_stats(reset=True)
    ctx.residual(dev(S), dev(Zi * 2.0 ** -20), "ozaki", D=D)
    names = {k["name"] for k in ctx.kernel_stats()}
    ctx.set_profiling(False)
    assert ("tc_gemm.crt" if ctx.emu == "auto" else "tc_gemm.ozaki") in names, names
    assert np.array_equal(D[:, cols].cpu().numpy(), np.eye(n)[:, cols] - X)


@pytest.mark.parametrize("n", [700, 2100])
def test_residual_exact_with_norm_bound_moduli(ctx, n):
    """Rows far from the worst case: Z = 2^-10 (I + sparse integers), S an integer matrix with
    64 on the diagonal and sparse small entries off it.  Every row's scaled 2-norm is about 1/2
    (one dominant entry), so by Cauchy-Schwarz the integer products need about log2(N) bits fewer
    than the bound N 2^(2T) that holds for any rows: 14 moduli instead of 16.  d must still equal
    I - Z^T S Z bit for bit, and the tensor-core flops show how many moduli ran (k 2 N^3 for Z^T S,
    k N^3 for the symmetric Z^T A)."""
    import torch
    g = np.random.default_rng(100 + n)
    Zi = np.eye(n) * 1024.0
    m = g.random((n, n)) < 0.02
    Zi[m] += g.integers(-3, 4, m.sum())
    A = np.where(g.random((n, n)) < 0.02, g.integers(-2, 3, (n, n)), 0).astype(np.float64)
    S = A + A.T
    np.fill_diagonal(S, 64.0)
    X = Zi.T @ (S @ Zi)
    assert np.abs(X).max() < 2.0 ** 40
    d_exact = np.eye(n) - X * 2.0 ** -40
    D = torch.empty((n, n), dtype=torch.float64, device="cuda")
    ctx.set_profiling(True)
    ctx.kernel_stats(reset=True)
    ctx.residual(dev(S), dev(Zi * 2.0 ** -20), "ozaki", D=D)
    stats = {k["name"]: k for k in ctx.kernel_stats()}
    ctx.set_profiling(False)
    assert np.array_equal(D.cpu().numpy(), d_exact)
    if ctx.emu == "auto":
        k = stats["tc_gemm.crt"]["flops"] / (3.0 * n ** 3)
        assert stats["tc_gemm.crt"]["launches"] == 2 and abs(k - round(k)) < 1e-9, stats["tc_gemm.crt"]
        assert round(k) == 14, k


def test_ozaki_residual_unaligned_operand_bit_identical(ctx):
    """S at an 8-byte offset (no 16-byte loads): the same digits, so the same bits as aligned S."""
    import torch
    n = 201
    S, Q, lam = synth.householder_spd(n, seed=7)
    Z = (Q * lam ** -0.5) @ Q.T + 1e-3 * np.random.default_rng(7).standard_normal((n, n))
    buf = torch.empty(n * n + 1, dtype=torch.float64, device="cuda")
    Su = buf[1:].view(n, n)
    Su.copy_(dev(S))
    assert Su.data_ptr() % 16 == 8
    D1 = torch.empty((n, n), dtype=torch.float64, device="cuda")
    D2 = torch.empty_like(D1)
    e1 = ctx.residual(dev(S), dev(Z), "ozaki", D=D1)
    e2 = ctx.residual(Su, dev(Z), "ozaki", D=D2)
    assert torch.equal(D1, D2) and e1 == e2


def test_ozaki_residual_of_exact_factor_is_tiny(ctx):
    """Z = S^{-1/2} from the generator's own factors: the FP64-accurate residual sits at the
    FP64 noise floor, far below anything FP32 accumulation could resolve."""
    n = 300
    S, Q, lam = synth.householder_spd(n, seed=77)
    Z = (Q * lam ** -0.5) @ Q.T
    err = ctx.residual(dev(S), dev(Z), "ozaki")
    _, err_or = oracle.residual(S, Z)
    # FP32 accumulation could not resolve anything below ~1e-6 here; the slicing truncation
    # (2^-54 normwise, s = 9 slices of 6 bits) leaves a floor within a few times FP64's
    assert err < 1e-12 and abs(err - err_or) < 1e-12


@pytest.mark.parametrize("prec", ["bf16", "bf16_split"])
def test_mixed_ozaki_refinement(ctx, prec):
    S, Q, lam = synth.householder_spd(256, seed=0)
    r = ctx.refine(dev(S), None, order=2, precision=prec, tol=1e-12, refine_mode="ozaki")
    Z = r.Z.cpu().numpy()
    _, e = oracle.residual(S, Z)
    assert e / 16.0 <= 1e-12
    assert abs(r.info["resid_f"] - e) <= 1e-12  # slicing noise floor, see module docstring
    assert r.info["refine_iters"] >= 1


@pytest.mark.parametrize("m", [3, 5])
def test_mixed_ozaki_higher_order(ctx, m):
    S, Q, lam = synth.householder_spd(190, seed=m)
    r = ctx.refine(dev(S), None, order=m, precision="bf16", tol=1e-12, refine_mode="ozaki")
    _, e = oracle.residual(S, r.Z.cpu().numpy())
    assert e / math.sqrt(190) <= 1e-12


def test_mixed_ozaki_workload2(ctx):
    S = synth.cubic_overlap()
    n = S.shape[0]
    r = ctx.refine(dev(S), None, order=2, precision="bf16", tol=1e-12, refine_mode="ozaki")
    assert r.info["resid_f"] / math.sqrt(n) <= 1e-12
    # the FP64 CUDA-core residual of the returned Z confirms it
    e = ctx.residual(dev(S), r.Z, "native")
    assert e / math.sqrt(n) <= 1e-12
    assert abs(e - r.info["resid_f"]) <= 1e-12 * math.sqrt(n)


def test_ozaki_residual_ill_conditioned_many_slices(ctx):
    """cond ~1e5 with max|Z| ~ 300: the slice count grows past ten (128-bit fixed-point slicing);
    the residual must still match the FP64 oracle normwise."""
    import torch
    n = 600
    S, Q, lam = synth.householder_spd(n, seed=91, lam_lo=1e-5, lam_hi=1.0)
    g = np.random.default_rng(91)
    Z = (Q * lam ** -0.5) @ Q.T + 1e-6 * g.standard_normal((n, n))
    assert np.max(np.abs(Z)) ** 2 * np.max(np.abs(S).sum(axis=1)) > 2.0 ** 13   # more than 11 slices
    d_or, err_or = oracle.residual(S, Z)
    D = torch.empty((n, n), dtype=torch.float64, device="cuda")
    err = ctx.residual(dev(S), dev(Z), "ozaki", D=D)
    scale = np.max(np.abs(Z).T @ np.abs(S) @ np.abs(Z))
    assert np.max(np.abs(D.cpu().numpy() - d_or)) <= 1e-13 * scale
    assert abs(err - err_or) <= 1e-13 * scale * n
