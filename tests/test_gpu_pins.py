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


def _first_ratio_above_one(hist):
    """Fig. 1's index (reading 16): the paper plots Err_{n+1} / Err_n^3 at n = 0, 1, ...; the first n
    whose ratio exceeds one."""
    for n in range(len(hist) - 1):
        if hist[n + 1] > hist[n] ** 3:
            return n
    return None


def test_paper_synthetic_fp64_path_matches_oracle_n1024(ctx):
    """Sec. 5.1's S~ at N = 1024 from Z0 = S^{-1/2} + 0.005 U: the FP64 GPU path against the oracle's
    Algorithm 2 with the same number of updates (spec tolerance 1e-12), and the history of the
    oracle's own stop."""
    n = 1024
    S = synth.paper_synthetic(n)
    w, V = np.linalg.eigh(S)
    Z0 = (V * w ** -0.5) @ V.T + synth.random_warm_start(n, 0.005)
    Zo, ho, ito = oracle.refine(S, Z0, m=2, nmax=50)
    r = ctx.refine(dev(S), dev(Z0), order=2, precision="fp64", fixed_iters=ito)
    Z = r.Z.cpu().numpy()
    assert np.linalg.norm(Z - Zo) / np.linalg.norm(Zo) <= 1e-12
    for h, hh in zip(r.hist[:ito + 1], ho):
        if hh > 1e-12:
            assert abs(h - hh) <= 1e-9 * hh
    # under its own stop rule the GPU path stops within one update of the oracle
    r2 = ctx.refine(dev(S), dev(Z0), order=2, precision="fp64")
    assert abs(r2.info["iters"] - ito) <= 1


def test_paper_synthetic_n16384_iterations_and_fig1_ratio(ctx, golden):
    """Sec. 5.3 and Fig. 1 at N = 16384: S~ (reading 8), Z0 = S^{-1/2} + 0.005 U, the split scheme
    (h)(h)+(h)(l)+(l)(h) under Algorithm 2's stop.  The paper reports 5 iterations and a Frobenius
    stop ratio first above one at n = 4 (A100; its rounding and seed differ, so both +-1)."""
    import torch
    n = 16384
    S = synth.paper_synthetic_torch(n)
    Z0 = synth.paper_start_torch(S, 0.005, seed=0)
    r = ctx.refine(S, Z0, order=2, precision="fp16_split", refine_steps=0, final_residual=0)
    hist = [float(h) for h in r.hist]
    ref = golden["iterations_paper_synthetic"]["value"]["16384"]
    assert abs(r.info["iters"] - ref) <= 1, (r.info, hist)
    first = _first_ratio_above_one(hist[:r.info["iters"] + 1])
    assert first is not None and abs(first - 4) <= 1, hist
    # cubic decay before the stop (Sec. 4.1, Eq. stopL2): every accepted step satisfied the bound
    assert all(hist[k] <= hist[k - 1] ** 3 for k in range(1, r.info["iters"]))
    del S, Z0
    torch.cuda.empty_cache()
