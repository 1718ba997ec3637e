"""Wide CRT residues (zfact_set_emulation("wide")): FP64-accurate products whose operand rows
need more than the sixteen moduli hold (an ill-conditioned Z: 60 to 83 bits per row), formed
modulo up to 24 moduli with a six-limb reconstruction, against the FP64 oracle.

The bit-exact cases use integer S and Z = Z_int 2^-k: every entry of S Z, Z^T S and
Z^T S Z is an integer multiple of a power of two that FP64 holds, the rows' fixed point
keeps every bit, and the CRT bound covers the integer products, so d must equal
I - Z^T S Z exactly.  The scale 2^-k sets max|Z|^2 g_hi and with it the bits per row
(66 to 78 here), which the kernel list confirms went through the wide residues."""
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
    c.set_emulation("wide")
    yield c
    c.close()


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _residual_with_stats(ctx, S, Z, D):
    ctx.set_profiling(True)
    ctx.kernel_stats(reset=True)
    err = ctx.residual(dev(S), dev(Z), "ozaki", D=D)
    names = {k["name"] for k in ctx.kernel_stats()}
    ctx.set_profiling(False)
    return err, names


@pytest.mark.parametrize("n,k", [(300, 8), (520, 2), (4300, 8)])
def test_wide_residual_exact_on_scaled_integer_inputs(ctx, n, k):
    import torch
    g = np.random.default_rng(1000 + n + k)
    Zi = g.integers(-2 ** 8, 2 ** 8, (n, n)).astype(np.float64)
    A = g.integers(-8, 8, (n, n)).astype(np.float64)
    S = A + A.T
    Z = Zi * 2.0 ** -k
    cols = np.arange(n) if n <= 600 else np.unique(np.concatenate([g.choice(n, 24, replace=False), [0, n - 1]]))
    Xi = Zi.T @ (S @ Zi[:, cols])                  # integers below 2^53: exact in any order
    assert np.abs(Xi).max() < 2.0 ** 52
    X = Xi * 2.0 ** (-2 * k)
    D = torch.empty((n, n), dtype=torch.float64, device="cuda")
    err, names = _residual_with_stats(ctx, S, Z, D)
    assert "oz_crt.wide" in names and "tc_gemm.ozaki" not in names, names
    assert np.array_equal(D[:, cols].cpu().numpy(), np.eye(n)[:, cols] - X)
    if n <= 600:
        ref = np.linalg.norm(np.eye(n) - X)
        assert abs(err - ref) <= 1e-13 * ref


@pytest.mark.parametrize("n", [64, 257, 600])
def test_wide_residual_ill_conditioned_matches_oracle(ctx, n):
    """cond 1e5 with max|Z| ~ 300: more than 62 bits per row, past the sixteen moduli."""
    import torch
    S, Q, lam = synth.householder_spd(n, seed=91 + n, lam_lo=1e-5, lam_hi=1.0)
    g = np.random.default_rng(91 + n)
    Z = (Q * lam ** -0.5) @ Q.T + 1e-6 * g.standard_normal((n, n))
    assert np.max(np.abs(Z)) ** 2 * np.max(np.abs(S).sum(axis=1)) > 2.0 ** 13
    d_or, err_or = oracle.residual(S, Z)
    D = torch.empty((n, n), dtype=torch.float64, device="cuda")
    err, names = _residual_with_stats(ctx, S, Z, D)
    assert "oz_crt.wide" in names, names
    scale = np.max(np.abs(Z).T @ np.abs(S) @ np.abs(Z))
    assert np.max(np.abs(D.cpu().numpy() - d_or)) <= 1e-13 * scale
    assert abs(err - err_or) <= 1e-13 * scale * n


def test_wide_residual_large_z_n4300_matches_oracle(ctx):
    """N = 4300 (two K-chunks per residue product): the cubic overlap with Z = 16 (I + 1e-3 G), so
    max|Z|^2 g_hi ~ 2^8.5 asks for 66 bits per row; d element by element against the oracle."""
    import torch
    n = 4300
    S = synth.cubic_overlap(n_side=17)[:n, :n].copy()
    Z = 16.0 * (np.eye(n) + 1e-3 * np.random.default_rng(4300).standard_normal((n, n)))
    d_or, err_or = oracle.residual(S, Z)
    D = torch.empty((n, n), dtype=torch.float64, device="cuda")
    err, names = _residual_with_stats(ctx, S, Z, D)
    assert "oz_crt.wide" in names, names
    scale = float(np.max(np.abs(Z).T @ (np.abs(S) @ np.abs(Z))))
    assert float(np.max(np.abs(D.cpu().numpy() - d_or))) <= 1e-13 * scale
    assert abs(err - err_or) <= 1e-13 * scale * n


def test_wide_matches_slices_on_the_same_residual(ctx):
    """The wide residues and the error-free slices keep the same bits per row: on the same
    ill-conditioned input their d agree to the scale of FP64 rounding."""
    import torch
    from paper_2404_19163_gb300 import Context
    n = 400
    S, Q, lam = synth.householder_spd(n, seed=5, lam_lo=1e-5, lam_hi=1.0)
    Z = (Q * lam ** -0.5) @ Q.T
    D1 = torch.empty((n, n), dtype=torch.float64, device="cuda")
    _residual_with_stats(ctx, S, Z, D1)
    with Context(0) as c2:
        c2.set_emulation("slices")
        D2 = torch.empty_like(D1)
        c2.residual(dev(S), dev(Z), "ozaki", D=D2)
    scale = np.max(np.abs(Z).T @ np.abs(S) @ np.abs(Z))
    assert float((D1 - D2).abs().max()) <= 1e-13 * scale
