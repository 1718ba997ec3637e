"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each check below ties the oracle to something other than itself: constants
printed in the paper (tests/golden), closed forms, brute force on tiny inputs,
independent library routines (eigh, LU) and exact rational arithmetic.  The
``check_*`` helpers take the oracle functions as arguments so that
test_oracle_mutations.py can plant mistakes in them and see a pin fail.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2404_19163_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def F(s):
    return Fraction(s)


# ------------------------------------------------------------------ polynomial helpers (exact)
def pmul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def residual_map_in_t(c):
    """Coefficients (in t, X = 1 + t) of X p(d)^2 with d = I - X = -t,
    p(d) = sum_k c_k d^k: the scalar map of one iteration (Sec. 4.1)."""
    p = [ck * (-1) ** k for k, ck in enumerate(c)]      # p as a polynomial in t
    return pmul([Fraction(1), Fraction(1)], pmul(p, p))


def check_coefficients(coeffs_fn, golden):
    c = coeffs_fn(2)
    # Appendix A: a0 I + a1 X + a2 X^2; substituting X = 1 - d must give p(d).
    a = [F(v) for v in golden["a_m2"]["value"]]
    # sum_k a_k (1 - d)^k expanded in d
    from_a = [a[0] + a[1] + a[2], -a[1] - 2 * a[2], a[2]]
    assert list(c) == from_a, (c, from_a)
    # Sec. 4.1 / Appendix A: X_{n+1} = I + c t^3 + d t^4 + e t^5 for X_n = I + t.
    g = residual_map_in_t(c)
    cde = [F(v) for v in golden["cde_m2"]["value"]]
    assert g == [1, 0, 0] + cde, g
    assert sum(abs(x) for x in cde) == 1          # the bound of Eq. norm condition is < 1 for ||d|| < 1
    # nu_max = m + 1 for every order: the lowest non-zero error term is t^(m+1)
    for m in range(2, 6):
        g = residual_map_in_t(coeffs_fn(m))
        assert g[0] == 1 and all(x == 0 for x in g[1:m + 1]) and g[m + 1] != 0, (m, g)
    assert golden["nu_max_m2"]["value"] == 3


def test_coefficients_match_paper(golden):
    check_coefficients(oracle.coeffs, golden)


def test_c_coeffs_match_exact():
    import ctypes
    lib = oracle._load()
    for m in range(2, 6):
        buf = (ctypes.c_double * (m + 1))()
        lib.zo_coeffs(m, ctypes.cast(buf, ctypes.c_void_p))
        assert [buf[k] for k in range(m + 1)] == [float(x) for x in oracle.coeffs(m)]


# ------------------------------------------------------------------ dense kernels vs independent routines
def test_matmul_and_residual_brute_force():
    g = np.random.default_rng(1)
    for n in (1, 2, 5, 17):
        A = g.standard_normal((n, n))
        B = g.standard_normal((n, n))
        ref = [[math.fsum(A[i, k] * B[k, j] for k in range(n)) for j in range(n)] for i in range(n)]
        assert np.allclose(oracle.matmul(A, B), np.array(ref), rtol=1e-13, atol=1e-13)
        S = A @ A.T + n * np.eye(n)
        Z = 0.1 * g.standard_normal((n, n)) + np.eye(n) / math.sqrt(n)
        d, err = oracle.residual(S, Z)
        X = [[math.fsum(Z[k, i] * S[k, l] * Z[l, j] for k in range(n) for l in range(n))
              for j in range(n)] for i in range(n)]
        dref = np.eye(n) - np.array(X)
        assert np.allclose(d, dref, rtol=1e-12, atol=1e-12)
        assert np.array_equal(d, d.T)
        assert abs(err - math.sqrt(math.fsum(v * v for v in dref.ravel()))) < 1e-12 * max(1, err)


def test_poly_brute_force():
    g = np.random.default_rng(2)
    n = 6
    d = g.standard_normal((n, n)) * 0.1
    d = d + d.T
    for m in range(2, 6):
        c = [float(x) for x in oracle.coeffs(m)]
        ref = sum(c[k] * np.linalg.matrix_power(d, k) for k in range(1, m + 1))
        assert np.allclose(oracle.poly(d, m), ref, rtol=1e-14, atol=1e-15)


# ------------------------------------------------------------------ closed forms
def check_diagonal(refine_fn):
    """Diagonal S, Z0 = s I: every iterate is diagonal and follows the scalar
    recursion z <- z p(1 - lam z^2); the limit is S^{-1/2} exactly."""
    import mpmath as mp
    mp.mp.dps = 40
    g = np.random.default_rng(3)
    lam = np.exp(g.uniform(math.log(0.3), math.log(3.0), 12))
    S = np.diag(lam)
    s = 1.0 / math.sqrt(lam.max())
    Z, hist, it = refine_fn(S, np.eye(12) * s, m=2, nmax=50, fixed_iters=4)
    zs = [mp.mpf(s)] * 12
    for _ in range(4):
        zs = [z * (1 + (1 - l * z * z) / 2 + mp.mpf(3) / 8 * (1 - l * z * z) ** 2)
              for z, l in zip(zs, [mp.mpf(float(x)) for x in lam])]
    assert np.allclose(np.diag(Z), [float(z) for z in zs], rtol=1e-14, atol=0)
    assert np.count_nonzero(Z - np.diag(np.diag(Z))) == 0
    Zc, hist, it = refine_fn(S, np.eye(12) * s, m=2, nmax=50)
    assert np.allclose(np.diag(Zc), lam ** -0.5, rtol=2e-15, atol=0)


def test_diagonal_exact():
    check_diagonal(oracle.refine)


def check_two_by_two(refine_fn):
    """Block-diagonal [[1, b], [b, 1]] blocks: S^{-1/2} = 1/2 [[u+v, u-v], [u-v, u+v]],
    u = (1+b)^{-1/2}, v = (1-b)^{-1/2}; Z0 = s I converges to it."""
    bs = [0.0, 0.3, -0.45, 0.7, -0.8]
    n = 2 * len(bs)
    S = np.zeros((n, n))
    R = np.zeros((n, n))
    for k, b in enumerate(bs):
        S[2 * k:2 * k + 2, 2 * k:2 * k + 2] = [[1, b], [b, 1]]
        u, v = (1 + b) ** -0.5, (1 - b) ** -0.5
        R[2 * k:2 * k + 2, 2 * k:2 * k + 2] = 0.5 * np.array([[u + v, u - v], [u - v, u + v]])
    s = 1.0 / math.sqrt(1.8)
    Z, hist, it = refine_fn(S, np.eye(n) * s, m=2, nmax=50)
    assert np.linalg.norm(Z - R) / np.linalg.norm(R) < 1e-14


def test_two_by_two_closed_form():
    check_two_by_two(oracle.refine)


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_tiny_random_spd_vs_lu(n):
    g = np.random.default_rng(100 + n)
    for trial in range(5):
        Qm, _ = np.linalg.qr(g.standard_normal((n, n)))
        lam = np.exp(g.uniform(0, math.log(1e3), n))
        S = (Qm * lam) @ Qm.T
        S = 0.5 * (S + S.T)
        Z, hist, it = oracle.refine(S, None, m=2, nmax=100)
        assert it > 0
        lu = scipy.linalg.lu_factor(S)
        Sinv = scipy.linalg.lu_solve(lu, np.eye(n))
        assert np.linalg.norm(Z @ Z.T - Sinv) / np.linalg.norm(Sinv) < 1e-12
        assert np.linalg.norm(Z.T @ S @ Z - np.eye(n)) < 1e-13 * 1e3


def test_householder_closed_form():
    """Workload 1: S^{-1/2} = Q diag(lam^{-1/2}) Q^T from the generator's own factors."""
    S, Q, lam = synth.householder_spd(64, seed=0)
    R = (Q * lam ** -0.5) @ Q.T
    Z, hist, it = oracle.refine(S, None, m=2, nmax=50)
    assert np.linalg.norm(Z - R) / np.linalg.norm(R) < 1e-13
    # Algorithm 2 stopped when the cube test (or the monotone guard) fired
    assert hist[it] > hist[it - 1] ** 3 or hist[it] >= hist[it - 1]
    assert all(hist[i] <= hist[i - 1] ** 3 for i in range(1, it))


def check_scalar_map(refine_fn):
    """Any Z0: eig(X_n) = g^n(eig(X0)), so the residual history follows from
    the spectrum of X0 alone (mpmath), down to the FP64 noise floor."""
    g = np.random.default_rng(7)
    n = 24
    S, Q, lam = synth.householder_spd(n, seed=3)
    Z0 = (Q * lam ** -0.5) @ Q.T + 0.05 * g.standard_normal((n, n))   # general, non-symmetric
    X0 = Z0.T @ S @ Z0
    mu = np.linalg.eigvalsh(0.5 * (X0 + X0.T))
    assert np.all(np.abs(1 - mu) < 1)
    for m in (2, 3, 5):
        Z, hist, it = refine_fn(S, Z0, m=m, nmax=50, fixed_iters=3)
        pred = oracle.scalar_map_hist(mu, m, 3)
        for h, p in zip(hist, pred):
            if p > 1e-9:
                assert abs(h - p) <= 1e-9 * p + 1e-12, (m, hist, pred)


def test_scalar_map_history():
    check_scalar_map(oracle.refine)


def test_warm_start_limit():
    """Z_n = Z0 F_n(X0) with F_n(x) -> x^{-1/2}: the limit is Z0 X0^{-1/2}."""
    g = np.random.default_rng(8)
    n = 20
    S, Q, lam = synth.householder_spd(n, seed=4)
    Z0 = (Q * lam ** -0.5) @ Q.T + 0.03 * g.standard_normal((n, n))
    X0 = Z0.T @ S @ Z0
    w, V = np.linalg.eigh(0.5 * (X0 + X0.T))
    lim = Z0 @ ((V * w ** -0.5) @ V.T)
    Z, hist, it = oracle.refine(S, Z0, m=2, nmax=50)
    assert np.linalg.norm(Z - lim) / np.linalg.norm(lim) < 1e-13


# ------------------------------------------------------------------ the stop rule (Sec. 4.1, Algorithm 2)
# The stop iteration is predicted without the oracle: the exact residual history E_n comes from
# the scalar map on eig(X0) (mpmath), and the computed Err_n is only assumed to lie in an interval
# around E_n:
#   E_n >= 1e-9: within 1e-9 E_n + 1e-12 (the agreement check_scalar_map asserts);
#   E_n <  1e-9: in [max(PHI_LO, E_n - ETA), E_n + ETA], ETA a generous FP64 noise level for these
#   N <= 64, cond <= 25 cases, and PHI_LO below one unit in the last place of 1 (2^-53): a computed
#   d = I - X with any diagonal entry X_ii != 1 has |d_ii| >= 2^-53 (checked on the result below).
# Rule (Algorithm 2 with reading 2's guard): stop after update n when Err_n > Err_{n-1}^3 or
# Err_n >= Err_{n-1}.  A step is predicted only when every value in the intervals gives the same
# answer; the inputs are chosen so that every step is determinate.
STOP_PHI_LO, STOP_ETA = 1e-17, 1e-13


def _stop_interval(E):
    if E >= 1e-9:
        t = 1e-9 * E + 1e-12
        return E - t, E + t
    return max(STOP_PHI_LO, E - STOP_ETA), E + STOP_ETA


def predict_stop(mu, m=2, nmax=12):
    """(n, which test fired) from the spectrum mu of X0 alone; n = None if a step is ambiguous."""
    E = oracle.scalar_map_hist(mu, m, nmax)
    for n in range(1, nmax + 1):
        alo, ahi = _stop_interval(E[n - 1])
        blo, bhi = _stop_interval(E[n])
        cube_yes, cube_no = blo > ahi ** 3, bhi <= alo ** 3
        guard_yes, guard_no = blo >= ahi, bhi < alo
        if cube_yes:
            return n, "cube"
        if guard_yes:
            return n, "guard"
        if not (cube_no and guard_no):
            return None, n
    return None, "nmax"


def _start_with_spectrum(n, seed, mu):
    """Z0 = Q diag(sqrt(mu/lam)) Q^T, so X0 = Z0^T S Z0 = Q diag(mu) Q^T (S = Q diag(lam) Q^T)."""
    S, Q, lam = synth.householder_spd(n, seed=seed)
    return S, (Q * np.sqrt(mu / lam)) @ Q.T


def stop_cases():
    n = 32
    # (a) the cube test fires at the FP64 floor: E_1 ~ 1e-6, so E_1^3 ~ 1e-18 lies below any
    #     non-zero computed Err_2 while E_1^2 ~ 1e-12 lies above it (a squared test would go on)
    mu_a = np.concatenate([[1.0 - 0.0117], np.full(n - 1, 1.0 - 1e-3)])
    # (b) Err_0 >= 1 and the iteration diverges (an eigenvalue of X0 at 3 maps to 6.75): Err grows
    #     but by less than its cube, so only the monotone guard stops it
    mu_b = np.linspace(0.3, 3.0, n)
    cases = [("cube_at_floor", *_start_with_spectrum(n, 3, mu_a), 2, "cube"),
             ("monotone_guard", *_start_with_spectrum(n, 3, mu_b), 1, "guard")]
    # (c) cold starts (Gershgorin-scaled identity, workload 1's generator)
    for nn, seed in ((32, 4), (40, 1), (64, 0)):
        S, Q, lam = synth.householder_spd(nn, seed=seed)
        cases.append(("cold_%d_%d" % (nn, seed), S, None, None, "cube"))
    return cases


def check_stop_rule(refine_fn):
    for name, S, Z0, expect_n, expect_kind in stop_cases():
        n = S.shape[0]
        Zs = Z0 if Z0 is not None else np.eye(n) / math.sqrt(np.max(np.abs(S).sum(axis=1)))
        X0 = Zs.T @ S @ Zs
        mu = np.linalg.eigvalsh(0.5 * (X0 + X0.T))
        pred, kind = predict_stop(mu)
        assert pred is not None, (name, kind)          # the input must give a determinate prediction
        assert kind == expect_kind, (name, kind)
        if expect_n is not None:
            assert pred == expect_n, (name, pred)
        Z, hist, it = refine_fn(S, Z0, m=2, nmax=50)
        assert it == pred, (name, it, pred, hist)
        if kind == "cube":
            # premise of PHI_LO: the returned iterate's computed d has a non-zero diagonal entry
            d = np.eye(n) - Z.T @ S @ Z
            assert np.max(np.abs(np.diag(d))) > 0.0, name


def test_stop_rule_predicted_from_scalar_map():
    check_stop_rule(oracle.refine)


def test_algorithm1_tolerance_rule():
    S, Q, lam = synth.householder_spd(32, seed=5)
    Z, hist, it = oracle.refine(S, None, m=2, nmax=50, rule=1, tol=1e-6)
    assert hist[it] / math.sqrt(32) <= 1e-6
    assert hist[it - 1] / math.sqrt(32) > 1e-6


def test_gershgorin_scale():
    S = np.array([[2.0, -1.0, 0.5], [-1.0, 3.0, 0.25], [0.5, 0.25, 1.0]])
    assert oracle.gershgorin_scale(S) == 1.0 / math.sqrt(4.25)
    S, Q, lam = synth.householder_spd(40, seed=6)
    s = oracle.gershgorin_scale(S)
    mu = s * s * lam
    assert mu.max() <= 1.0 and mu.min() > 0.0


def test_alg3_refinement_extends_history():
    S, Q, lam = synth.householder_spd(32, seed=9)
    Z, hist, it = oracle.refine_alg3(S, None, m=2, refine_steps=1)
    assert len(hist) == it + 2
    assert hist[-1] < 1e-13


# ------------------------------------------------------------------ the hi/lo split (Sec. 3.1)
def test_split_bound_fp16(golden):
    assert golden["split_bound_fp16"]["value"] == "2^-22"
    g = np.random.default_rng(11)
    vals = np.concatenate([
        g.standard_normal(200000) * 10.0 ** g.uniform(-4, 4, 200000),
        [1.0, -1.0, 65504.0, 2.0 ** -14, 1 + 2.0 ** -11, 1 + 2.0 ** -12, 3.0, 1.0 / 3.0, 0.1],
    ])
    vals = vals[(np.abs(vals) >= 2.0 ** -3) & (np.abs(vals) <= 60000)]   # lo stays in FP16's normal range
    a32 = vals.astype(np.float32).astype(np.float64)
    hi, lo = oracle.split16(a32, "fp16")
    err = np.abs(a32 - hi.astype(np.float64) - lo.astype(np.float64))
    assert np.all(err <= 2.0 ** -22 * np.abs(a32))
    # hi is the nearest FP16 value (brute force against both neighbours)
    h16 = hi.astype(np.float16)
    up = np.nextafter(h16, np.float16(np.inf)).astype(np.float64)
    dn = np.nextafter(h16, np.float16(-np.inf)).astype(np.float64)
    assert np.all(np.abs(a32 - hi) <= np.abs(a32 - up)) and np.all(np.abs(a32 - hi) <= np.abs(a32 - dn))


def test_split_bound_bf16():
    g = np.random.default_rng(12)
    vals = g.standard_normal(100000) * 10.0 ** g.uniform(-10, 10, 100000)
    a32 = vals.astype(np.float32).astype(np.float64)
    hi, lo = oracle.split16(a32, "bf16")
    err = np.abs(a32 - hi.astype(np.float64) - lo.astype(np.float64))
    assert np.all(err <= 2.0 ** -16 * np.abs(a32))
    # BF16 values are FP32 values with the low 16 bits clear
    assert np.all((hi.view(np.uint32) & 0xFFFF) == 0) and np.all((lo.view(np.uint32) & 0xFFFF) == 0)
    # round to nearest even on the bit pattern
    bits = a32.astype(np.float32).view(np.uint32).astype(np.uint64)
    rne = ((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16) << 16
    assert np.array_equal(hi.view(np.uint32).astype(np.uint64), rne)


def test_split_power_of_two_scale_exact():
    g = np.random.default_rng(13)
    A = g.standard_normal(1000) * 1e-3
    h1, l1 = oracle.split16(A, "fp16", scale=2.0 ** 10)
    a32 = (A * 2.0 ** 10).astype(np.float32)
    assert np.array_equal(h1, a32.astype(np.float16).astype(np.float32))


# ------------------------------------------------------------------ features
def test_features_against_spectrum():
    S, Q, lam = synth.householder_spd(48, seed=10)
    f = oracle.features(S)
    rows = np.abs(S).sum(axis=1)
    dg = np.diag(S)
    g_hi = float(np.max(dg + (rows - np.abs(dg))))
    mu = lam / g_hi
    for k in range(1, 5):
        assert abs(f[6 + k] - np.mean((1 - mu) ** k)) < 1e-13
    assert abs(f[0] - math.log(48)) < 1e-15
    assert abs(f[1] - math.log(g_hi)) < 1e-13
    t1, t2 = np.mean(1 - mu), np.mean((1 - mu) ** 2)
    assert abs(f[12] - (t2 - t1 * t1)) < 1e-13
    assert abs(f[12] - np.var(1 - mu)) < 1e-13
    from scipy.stats import moment
    assert abs(f[13] - moment(1 - mu, 3)) < 1e-13
    assert abs(f[14] - moment(1 - mu, 4)) < 1e-13


def check_features_by_hand(features_fn):
    """All 16 features of a 3 x 3 S computed by hand.
    S = [[4,-1,0],[-1,3,1],[0,1,2]]: diagonal (4,3,2), absolute row sums (5,5,3) (signed: 3,3,3),
    off-diagonal sums (1,2,1), so g_hi = max(5,5,3) = 5 and g_lo = min(3,1,1) = 1.  d0 = I - S/5 =
    B/5 with B = [[1,1,0],[1,2,-1],[0,-1,3]]; B^2 = [[2,3,-1],[3,6,-5],[-1,-5,10]], so tr B = 6,
    tr B^2 = 18, tr B^3 = 5 + 20 + 35 = 60, tr B^4 = sum of (B^2)_ij^2 = 210, and
    t_k = tr(B^k) / (3 5^k): t1 = 2/5, t2 = 6/25, t3 = 4/25, t4 = 14/125.  ||d0||_F = sqrt(18)/5."""
    S = np.array([[4.0, -1.0, 0.0], [-1.0, 3.0, 1.0], [0.0, 1.0, 2.0]])
    t1, t2, t3, t4 = 0.4, 0.24, 0.16, 0.112
    want = [math.log(3), math.log(5), 1 / 5, 3 / 5, 2 / 5, 13 / 15, 3 / 5, t1, t2, t3, t4,
            math.sqrt(6) / 5, 0.08, 0.0, 0.0096, math.log(math.sqrt(18) / 5)]
    # the central moments by hand: t2 - t1^2 = 0.08; t3 - 3 t1 t2 + 2 t1^3 = 0.16 - 0.288 + 0.128;
    # t4 - 4 t1 t3 + 6 t1^2 t2 - 3 t1^4 = 0.112 - 0.256 + 0.2304 - 0.0768
    f = features_fn(S)
    assert len(f) == 16
    for k, (x, w) in enumerate(zip(f, want)):
        assert abs(x - w) <= 1e-14 * max(1.0, abs(w)), (k, x, w)


def test_features_by_hand():
    check_features_by_hand(oracle.features)


# ------------------------------------------------------------------ MLP
def test_gelu_values():
    from scipy.stats import norm
    x = np.array([-3.0, -1.0, 0.0, 0.5, 1.0, 2.0])
    assert np.allclose(oracle.gelu(x), x * norm.cdf(x), rtol=1e-15, atol=1e-16)
    assert abs(oracle.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15
    h = 1e-6
    assert np.allclose(oracle.gelu_grad(x), (oracle.gelu(x + h) - oracle.gelu(x - h)) / (2 * h), atol=1e-8)


def test_mlp_forward_hand_network():
    """W1 = [I_16; 0], W2 = I_64, W3 = e_0 (x) ones, zero biases:
    y0 = sum_i gelu(gelu(x_i)), logits 0."""
    P = np.zeros(oracle.mlp_num_params())
    (W1, b1), (W2, b2), (W3, b3) = oracle.mlp_unpack(P)
    W1[:16, :16] = np.eye(16)
    W2[:, :] = np.eye(64)
    W3[0, :] = 1.0
    x = np.random.default_rng(14).standard_normal((3, 16))
    y = oracle.mlp_forward(P, x)
    assert np.allclose(y[:, 0], oracle.gelu(oracle.gelu(x)).sum(axis=1), rtol=1e-14)
    assert np.all(y[:, 1:] == 0)


def check_mlp_gradient(backward_fn):
    g = np.random.default_rng(15)
    P = g.standard_normal(oracle.mlp_num_params()) * 0.3
    x = g.standard_normal((5, 16))
    ys = g.standard_normal(5)
    yo = g.integers(0, 4, 5)
    grad = backward_fn(P, x, ys, yo, 0.7)
    idx = g.choice(P.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        Pp = P.copy(); Pp[i] += h
        Pm = P.copy(); Pm[i] -= h
        fd = (oracle.mlp_loss(Pp, x, ys, yo, 0.7) - oracle.mlp_loss(Pm, x, ys, yo, 0.7)) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_mlp_gradient_finite_differences():
    check_mlp_gradient(oracle.mlp_backward)


def test_adam_first_step_is_sign():
    g = np.random.default_rng(16)
    P = g.standard_normal(50)
    G = g.standard_normal(50)
    P1, m, v = oracle.adam_step(P, G, np.zeros(50), np.zeros(50), 1, lr=1e-2, eps=0.0)
    assert np.allclose(P1 - P, -1e-2 * np.sign(G), rtol=1e-12)


# ------------------------------------------------------------------ congruence transform (Sec. 2)
def check_congruence_exact(cong_fn):
    """Brute force in exact rational arithmetic on a tiny non-symmetric Z and symmetric H."""
    g = np.random.default_rng(11)
    n = 5
    Z = g.standard_normal((n, n))
    B = g.standard_normal((n, n))
    H = B + B.T
    Hp = cong_fn(H, Z)
    Zf = [[Fraction(float(v)) for v in r] for r in Z]
    Hf = [[Fraction(float(v)) for v in r] for r in H]
    for i in range(n):
        for j in range(n):
            ex = sum(Zf[k][i] * Hf[k][l] * Zf[l][j] for k in range(n) for l in range(n))
            mag = sum(abs(Zf[k][i] * Hf[k][l] * Zf[l][j]) for k in range(n) for l in range(n))
            assert abs(Fraction(float(Hp[i, j])) - ex) <= Fraction(2.0 ** -50) * mag, (i, j)


def check_congruence_generalized_eigs(cong_fn):
    """With Z Z^T = S^-1 (here Z = S^-1/2 from the generator's own factors), Z^T H Z has the
    eigenvalues of the generalized problem H c = e S c (Sec. 2): compare with LAPACK's sygv."""
    n = 60
    S, Q, lam = synth.householder_spd(n, seed=3)
    Z = (Q * lam ** -0.5) @ Q.T
    B = np.random.default_rng(4).standard_normal((n, n))
    H = B + B.T
    Hp = cong_fn(H, Z)
    assert np.array_equal(Hp, Hp.T)
    e_gen = scipy.linalg.eigh(H, S, eigvals_only=True)
    e = np.linalg.eigvalsh(Hp)
    assert np.allclose(e, e_gen, rtol=0, atol=1e-11 * np.max(np.abs(e_gen))), np.max(np.abs(e - e_gen))
    # H = S: the transform of the overlap itself is the identity (Eq. Def_Z)
    assert np.max(np.abs(cong_fn(S, Z) - np.eye(n))) <= 1e-12


def test_congruence_exact():
    check_congruence_exact(oracle.congruence)


def test_congruence_generalized_eigenvalues():
    check_congruence_generalized_eigs(oracle.congruence)
