"""The congruence transform H_perp = Z^T H Z (Sec. 2, Eq. standard_form) through zfact_congruence:
parity with the oracle, the generalized-eigenvalue property it exists for, and host operands."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2404_19163_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["auto", "slices"])
def ctx(request):
    """Both FP64-accurate product schemes: CRT residues (the default) and error-free slices."""
    from paper_2404_19163_gb300 import Context, build
    build.build()
    oracle.build()
    c = Context(0)
    c.set_emulation(request.param)
    yield c
    c.close()


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def case(n, seed):
    g = np.random.default_rng(seed)
    Z = g.standard_normal((n, n)) / np.sqrt(n) + np.eye(n)
    B = g.standard_normal((n, n))
    H = (B + B.T) / 2
    return H, Z


@pytest.mark.parametrize("n", [5, 200, 777, 1500])
@pytest.mark.parametrize("mode", ["native", "ozaki"])
def test_congruence_fp64_matches_oracle(ctx, n, mode):
    H, Z = case(n, n)
    ref = oracle.congruence(H, Z)
    got = ctx.congruence(dev(H), dev(Z), "fp64", mode).cpu().numpy()
    scale = np.max(np.abs(Z).T @ np.abs(H) @ np.abs(Z))
    assert np.array_equal(got, got.T)
    assert np.max(np.abs(got - ref)) <= 1e-13 * scale, float(np.max(np.abs(got - ref)) / scale)


@pytest.mark.parametrize("prec,tol", [("bf16_split", 2.0 ** -13), ("bf16", 2.0 ** -6)])
def test_congruence_bf16_matches_oracle(ctx, prec, tol):
    """BF16 hi/lo operands carry a relative error <= 2^-16 each (hi/lo split of Eq. splitStyle with
    8-bit significands), Z^T H is re-split once, and FP32 accumulation adds 2^-24 per term: four
    2^-16 sources and headroom give 2^-13 of |Z|^T |H| |Z| elementwise.  Plain BF16 (2^-8 per
    operand): 2^-6."""
    n = 1000
    H, Z = case(n, 5)
    ref = oracle.congruence(H, Z)
    got = ctx.congruence(dev(H), dev(Z), prec).cpu().numpy()
    scale = np.abs(Z).T @ np.abs(H) @ np.abs(Z)
    assert np.array_equal(got, got.T)
    assert np.all(np.abs(got - ref) <= tol * scale)


def test_congruence_gives_generalized_eigenvalues(ctx):
    """Z from this library's own factorization of S: eig(Z^T H Z) are the generalized
    eigenvalues of (H, S) from LAPACK's sygv."""
    n = 400
    S, Q, lam = synth.householder_spd(n, seed=9)
    r = ctx.refine(dev(S), None, order=2, precision="fp64")
    H, _ = case(n, 10)
    Hp = ctx.congruence(dev(H), r.Z, "fp64", "ozaki").cpu().numpy()
    e = np.linalg.eigvalsh(Hp)
    e_gen = scipy.linalg.eigh(H, S, eigvals_only=True)
    assert np.max(np.abs(e - e_gen)) <= 1e-11 * np.max(np.abs(e_gen))


def test_congruence_host_operands_identical(ctx):
    H, Z = case(300, 12)
    Hp_host = np.empty_like(H)
    ctx.congruence(np.ascontiguousarray(H), np.ascontiguousarray(Z), "fp64", "ozaki", Hp=Hp_host)
    Hp_dev = ctx.congruence(dev(H), dev(Z), "fp64", "ozaki").cpu().numpy()
    assert np.array_equal(Hp_host, Hp_dev)


def test_congruence_unsupported_precision(ctx):
    from paper_2404_19163_gb300.zfact import ZfactError
    H, Z = case(64, 13)
    with pytest.raises(ZfactError) as ei:
        ctx.congruence(dev(H), dev(Z), "fp16_split")
    assert ei.value.code == 7
