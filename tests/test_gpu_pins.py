"""GPU results against what the paper and the mathematics fix (independent of the CPU oracle's
dense loops): the scalar-map residual history, closed forms, and the paper's own synthetic
test matrix (Sec. 5.1) with its reported iteration counts."""
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


@pytest.mark.parametrize("m", [2, 3, 5])
def test_fp64_history_follows_scalar_map(ctx, m):
    g = np.random.default_rng(70 + m)
    n = 120
    S, Q, lam = synth.householder_spd(n, seed=70 + m)
    Z0 = (Q * lam ** -0.5) @ Q.T + 0.03 * g.standard_normal((n, n))
    X0 = Z0.T @ S @ Z0
    mu = np.linalg.eigvalsh(0.5 * (X0 + X0.T))
    r = ctx.refine(dev(S), dev(Z0), order=m, precision="fp64", fixed_iters=3)
    pred = oracle.scalar_map_hist(mu, m, 3)
    for h, p in zip(r.hist, pred):
        if p > 1e-9:
            assert abs(h - p) <= 1e-9 * p + 1e-12, (r.hist, pred)


@pytest.mark.parametrize("prec", ["fp64", "bf16_split", "fp16_split"])
def test_diagonal_s_gives_inverse_square_root(ctx, prec):
    lam = np.exp(np.random.default_rng(9).uniform(math.log(0.2), math.log(5.0), 300))
    r = ctx.refine(dev(np.diag(lam)), None, order=2, precision=prec, tol=1e-12)
    Z = r.Z.cpu().numpy()
    assert np.max(np.abs(np.diag(Z) - lam ** -0.5) / lam ** -0.5) <= 1e-12
    assert np.max(np.abs(Z - np.diag(np.diag(Z)))) <= 1e-12


def test_two_by_two_blocks_closed_form(ctx):
    bs = np.random.default_rng(10).uniform(-0.85, 0.85, 64)
    n = 128
    S = np.zeros((n, n))
    R = np.zeros((n, n))
    for k, b in enumerate(bs):
        S[2 * k:2 * k + 2, 2 * k:2 * k + 2] = [[1, b], [b, 1]]
        u, v = (1 + b) ** -0.5, (1 - b) ** -0.5
        R[2 * k:2 * k + 2, 2 * k:2 * k + 2] = 0.5 * np.array([[u + v, u - v], [u - v, u + v]])
    r = ctx.refine(dev(S), None, order=2, precision="fp64")
    assert np.linalg.norm(r.Z.cpu().numpy() - R) / np.linalg.norm(R) <= 1e-13


def test_paper_synthetic_matrix_iteration_count(ctx, golden):
    """Sec. 5.1/5.3: S~ symmetrised and shifted to lambda_min = 0.5, Z0 = S^{-1/2} + 0.005 U; the
    paper reports convergence in 3 iterations at N = 1024 (A100, split scheme).  The seed and the
    hardware rounding differ, so this is a +-1 check."""
    n = 1024
    S = synth.paper_synthetic(n)
    w, V = np.linalg.eigh(S)
    Zs = (V * w ** -0.5) @ V.T
    Z0 = Zs + synth.random_warm_start(n, 0.005)
    ref = golden["iterations_paper_synthetic"]["value"]["1024"]
    for prec in ("fp16_split", "fp64"):
        r = ctx.refine(dev(S), dev(Z0), order=2, precision=prec, refine_steps=0, final_residual=0)
        assert abs(r.info["iters"] - ref) <= 1, (prec, r.info, r.hist)
