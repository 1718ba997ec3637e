"""FP64 GPU path (the paper's "double") against the FP64 CPU oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_2404_19163_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2404_19163_gb300 import Context, build
    build.build()
    c = Context(0)
    yield c
    c.close()


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_workload1_fixed_iters_parity(ctx):
    S, Q, lam = synth.householder_spd(256, seed=0)
    Zo, ho, it = oracle.refine(S, None, m=2, nmax=50)
    r = ctx.refine(dev(S), None, order=2, precision="fp64", fixed_iters=it)
    assert rel(r.Z.cpu().numpy(), Zo) <= 1e-12
    assert np.allclose(r.hist[:it + 1], ho[:it + 1], rtol=1e-9, atol=1e-14)
    assert r.info["iters"] == it


def test_workload1_stop_rule(ctx):
    S, Q, lam = synth.householder_spd(256, seed=0)
    Zo, ho, it = oracle.refine(S, None, m=2, nmax=50)
    r = ctx.refine(dev(S), None, order=2, precision="fp64")
    # the stop fires at the FP64 noise floor; the count may differ by one there
    assert abs(r.info["iters"] - it) <= 1
    assert rel(r.Z.cpu().numpy(), Zo) <= 1e-12
    R = (Q * lam ** -0.5) @ Q.T
    assert rel(r.Z.cpu().numpy(), R) <= 1e-13
    assert r.info["resid_f"] / 16.0 < 1e-14


@pytest.mark.parametrize("n", [1, 7, 63, 65, 130, 300])
def test_ragged_sizes(ctx, n):
    S, Q, lam = synth.householder_spd(n, seed=n)
    Zo, ho, it = oracle.refine(S, None, m=2, nmax=50, fixed_iters=4)
    r = ctx.refine(dev(S), None, order=2, precision="fp64", fixed_iters=4)
    assert rel(r.Z.cpu().numpy(), Zo) <= 1e-12


@pytest.mark.parametrize("m", [3, 4, 5])
def test_higher_orders(ctx, m):
    S, Q, lam = synth.householder_spd(200, seed=m)
    Zo, ho, it = oracle.refine(S, None, m=m, nmax=50, fixed_iters=3)
    r = ctx.refine(dev(S), None, order=m, precision="fp64", fixed_iters=3)
    assert rel(r.Z.cpu().numpy(), Zo) <= 1e-12
    assert np.allclose(r.hist, ho, rtol=1e-9, atol=1e-14)


def test_warm_start_general_z0(ctx):
    g = np.random.default_rng(5)
    S, Q, lam = synth.householder_spd(150, seed=9)
    Z0 = (Q * lam ** -0.5) @ Q.T + 0.01 * g.standard_normal((150, 150))
    Zo, ho, it = oracle.refine(S, Z0, m=2, nmax=50, fixed_iters=3)
    r = ctx.refine(dev(S), dev(Z0), order=2, precision="fp64", fixed_iters=3)
    assert rel(r.Z.cpu().numpy(), Zo) <= 1e-12


def test_host_pointers(ctx):
    S, Q, lam = synth.householder_spd(100, seed=11)
    Zo, ho, it = oracle.refine(S, None, m=2, nmax=50, fixed_iters=3)
    r = ctx.refine(np.ascontiguousarray(S), None, order=2, precision="fp64", fixed_iters=3)
    assert isinstance(r.Z, np.ndarray)
    assert rel(r.Z, Zo) <= 1e-12


def test_tolerance_rule(ctx):
    S, Q, lam = synth.householder_spd(128, seed=12)
    Zo, ho, it = oracle.refine(S, None, m=2, nmax=50, rule=1, tol=1e-8)
    r = ctx.refine(dev(S), None, order=2, precision="fp64", stop_rule=1, tol=1e-8)
    assert r.info["iters"] == it
    assert rel(r.Z.cpu().numpy(), Zo) <= 1e-12


def test_errors(ctx):
    import torch
    from paper_2404_19163_gb300 import ZfactError
    S = dev(np.eye(8))
    with pytest.raises(ZfactError) as e:
        ctx.refine(S, None, order=7)
    assert e.value.code == 1
    Sn = np.eye(8)
    Sn[2, 3] = Sn[3, 2] = np.nan
    with pytest.raises(ZfactError) as e:
        ctx.refine(dev(Sn), None, order=2, precision="fp64")
    assert e.value.code == 4
    # a non-contractive start is reported as a warning with a result
    r = ctx.refine(dev(np.eye(8) * 4.0), dev(np.eye(8)), order=2, precision="fp64", fixed_iters=1,
                   raise_on_error=False)
    assert r.status == 100


@pytest.mark.parametrize("mode", ["ozaki", "native"])
def test_nonfinite_inputs_to_step_calls(ctx, mode):
    """A NaN or Inf planted on the host in S, Z or H: the step-level residual and the congruence
    report ZFACT_ERR_NONFINITE (the FP64-accurate scheme's row scaling must not turn them into finite
    fixed-point values), and the context keeps working."""
    from paper_2404_19163_gb300 import ZfactError
    n = 70
    S, Q, lam = synth.householder_spd(n, seed=12)
    Z = (Q * lam ** -0.5) @ Q.T
    for bad_s, bad_z, val in ((True, False, np.nan), (False, True, np.inf), (False, True, -np.nan)):
        Sb, Zb = S.copy(), Z.copy()
        if bad_s:
            Sb[5, 9] = Sb[9, 5] = val
        if bad_z:
            Zb[n - 1, 3] = val
        with pytest.raises(ZfactError) as e:
            ctx.residual(dev(Sb), dev(Zb), mode)
        assert e.value.code == 4, (bad_s, bad_z, val)
        with pytest.raises(ZfactError) as e:
            ctx.congruence(dev(Sb), dev(Zb), "fp64", mode)
        assert e.value.code == 4
    with pytest.raises(ZfactError) as e:
        ctx.congruence(dev(S), dev(np.where(np.eye(n) > 0, np.nan, Z)), "bf16")
    assert e.value.code == 4
    # the context still works
    d_or, e_or = oracle.residual(S, Z)
    assert abs(ctx.residual(dev(S), dev(Z), mode) - e_or) <= 1e-12


def test_workload2_full_size_against_oracle(ctx):
    """N = 4096 cubic Gaussian overlap, the launch configuration the benchmark times."""
    S = synth.cubic_overlap()
    n = S.shape[0]
    r = ctx.refine(dev(S), None, order=2, precision="fp64")
    it = r.info["iters"]
    Zo, ho, ito = oracle.refine(S, None, m=2, nmax=50, fixed_iters=it)
    assert rel(r.Z.cpu().numpy(), Zo) <= 1e-12
    assert r.info["resid_f"] / math.sqrt(n) < 1e-13


def test_inputs_written_on_another_stream_are_ordered(ctx):
    """S produced by a long torch product on a non-default current stream, passed at once: the binding
    waits for that stream, so the factorization reads the finished S (the context works on its own
    stream, which is not ordered after torch's)."""
    import torch
    n = 1500
    side = torch.cuda.Stream()
    g = torch.Generator(device="cuda").manual_seed(3)
    with torch.cuda.stream(side):
        B = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
        S = B @ B.T / n
        for _ in range(6):          # keep the stream busy well past the call below
            S = 0.5 * (S + S @ S.T / torch.linalg.matrix_norm(S, 2))
        S.diagonal().add_(1.0)
        r = ctx.refine(S, None, order=2, precision="fp64")
    torch.cuda.synchronize()
    _, e = oracle.residual(S.cpu().numpy(), r.Z.cpu().numpy())
    assert abs(r.info["resid_f"] - e) <= 1e-12 and e / math.sqrt(n) <= 1e-12


def test_tolerance_not_reached_within_nmax(ctx):
    """A forced tiny nmax with an unreachable tolerance (Algorithm 1's rule): NOT_CONVERGED, with the
    history valid up to the failure."""
    S, Q, lam = synth.householder_spd(64, seed=4)
    r = ctx.refine(dev(S), None, order=2, precision="fp64", stop_rule=1, tol=1e-30, nmax=2,
                   raise_on_error=False)
    assert r.status == 5 and r.info["iters"] == 2 and len(r.hist) >= 3


def test_workspace_limit_fails_cleanly(ctx):
    """A workspace cap below what the call needs: NOMEM before allocating, the context still usable."""
    from paper_2404_19163_gb300 import Context, ZfactError
    S, Q, lam = synth.householder_spd(300, seed=6)
    with Context(0) as c2:
        c2.set_workspace_limit(1 << 20)
        with pytest.raises(ZfactError) as e:
            c2.refine(dev(S), None, order=2, precision="bf16_split")
        assert e.value.code == 3 and "workspace limit" in c2.last_error()
        c2.set_workspace_limit(0)
        r = c2.refine(dev(S), None, order=2, precision="bf16_split", tol=1e-12)
        assert r.info["resid_f"] / math.sqrt(300) <= 1e-12


def test_bounded_wait_times_out_and_context_survives(ctx):
    """The bounded mbarrier wait of the tensor-core kernels, on a barrier nothing arrives at, gives up
    and is reported as ZFACT_ERR_TIMEOUT; the next call on the same context works."""
    assert ctx.selftest_timeout() == 6
    assert "bounded device wait" in ctx.last_error()
    S, Q, lam = synth.householder_spd(128, seed=8)
    r = ctx.refine(dev(S), None, order=2, precision="bf16_split", tol=1e-12)
    assert r.status in (0, 100) and r.info["resid_f"] / math.sqrt(128) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "bf16_split", "fp16_split"])
def test_start_scale_is_the_cold_start_with_that_scale(ctx, precision):
    """zfact_opts.start_scale (a proposal's scale) starts from Z0 = s I on the cold-start path: FP64
    against the oracle from the same explicit Z0; the mixed precisions start from Err_0 = ||I - s^2 S||_F
    and converge to tol."""
    S, Q, lam = synth.householder_spd(300, seed=11)
    s0 = oracle.gershgorin_scale(S)
    s = 1.3 * s0
    if precision == "fp64":
        Zo, ho, it = oracle.refine(S, np.eye(300) * s, m=2, nmax=50, fixed_iters=5)
        r = ctx.refine(dev(S), None, order=2, precision="fp64", fixed_iters=5, start_scale=s)
        assert rel(r.Z.cpu().numpy(), Zo) <= 1e-12
        assert np.allclose(r.hist[:6], ho[:6], rtol=1e-9, atol=1e-14)
        # start_scale = 0 is the Gershgorin default
        r0 = ctx.refine(dev(S), None, order=2, precision="fp64", fixed_iters=3, start_scale=0.0)
        r1 = ctx.refine(dev(S), None, order=2, precision="fp64", fixed_iters=3)
        assert np.array_equal(r0.Z.cpu().numpy(), r1.Z.cpu().numpy())
    else:
        r = ctx.refine(dev(S), None, order=3, precision=precision, tol=1e-12, start_scale=s)
        _, err = oracle.residual(S, r.Z.cpu().numpy())
        assert err / math.sqrt(300) <= 1e-12
        e0 = np.linalg.norm(np.eye(300) - s * s * S)
        assert abs(r.hist[0] - e0) <= 1e-5 * e0


def test_start_scale_that_does_not_contract_falls_back(ctx):
    """A start scale s = 3 / sqrt(lambda_max) puts the largest eigenvalue of X0 = s^2 S at 9, where the
    iteration diverges: the bulk cannot contract, so the call starts again from the Gershgorin scale and
    still meets tol.  The returned history is the second run's (Err_0 = ||I - s0^2 S||_F)."""
    S, Q, lam = synth.householder_spd(300, seed=12)
    s0 = oracle.gershgorin_scale(S)
    r = ctx.refine(dev(S), None, order=2, precision="bf16_split", tol=1e-12, start_scale=3.0 / math.sqrt(lam.max()))
    assert r.status in (0, 100)   # 100: the Gershgorin start's ||I - X0||_F is above 1 (a warning)
    _, err = oracle.residual(S, r.Z.cpu().numpy())
    assert err / math.sqrt(300) <= 1e-12
    e0 = np.linalg.norm(np.eye(300) - s0 * s0 * S)
    assert abs(r.hist[0] - e0) <= 1e-5 * e0
