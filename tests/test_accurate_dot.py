"""Pins of the doubled-precision reference used to judge FP64-accurate residuals: every result is
compared with exact rational arithmetic."""
from fractions import Fraction

import numpy as np

import accurate_dot as ad

U = 2.0 ** -53


def exact_rows(A, x):
    return [sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(row, x)), Fraction(0)) for row in A]


def test_two_sum_two_prod_error_free():
    g = np.random.default_rng(0)
    a = g.standard_normal(500) * 10.0 ** g.integers(-20, 20, 500)
    b = g.standard_normal(500) * 10.0 ** g.integers(-20, 20, 500)
    s, e = ad.two_sum(a, b)
    p, f = ad.two_prod(a, b)
    for k in range(500):
        assert Fraction(s[k]) + Fraction(e[k]) == Fraction(a[k]) + Fraction(b[k])
        assert Fraction(p[k]) + Fraction(f[k]) == Fraction(a[k]) * Fraction(b[k])


def test_matvec_dd_under_cancellation():
    """Rows built to cancel by ~30 orders of magnitude: the pair (hi, lo) still matches the exact
    sum to u^2 of the terms, where a plain FP64 sum loses every digit."""
    g = np.random.default_rng(1)
    n, m = 24, 301
    A = g.standard_normal((n, m)) * 10.0 ** g.integers(-8, 8, (n, m))
    x = g.standard_normal(m)
    # make each row's leading terms cancel: append the negated FP64 row sum split over two columns
    A = np.concatenate([A, np.zeros((n, 2))], axis=1)
    x = np.concatenate([x, [1.0, 1.0]])
    for i in range(n):
        t = float(sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(A[i, :m], x[:m])))
        A[i, m] = -t
    ex = exact_rows(A, x)
    hi, lo = ad.matvec_dd(A, x, block=7)
    plain_lost = 0
    for i in range(n):
        mag = sum(abs(Fraction(float(a)) * Fraction(float(b))) for a, b in zip(A[i], x))
        got = Fraction(hi[i]) + Fraction(lo[i])
        assert abs(got - ex[i]) <= Fraction(U * U) * mag * 20 + Fraction(U) * abs(ex[i]), i
        if abs(Fraction(float(A[i] @ x)) - ex[i]) > Fraction(2 * U) * abs(ex[i]):
            plain_lost += 1
    assert plain_lost > n // 2  # the case is a real test: plain FP64 fails it


def test_residual_column_exact():
    g = np.random.default_rng(2)
    n = 33
    B = g.standard_normal((n, n))
    S = B @ B.T / n + np.eye(n)
    w, V = np.linalg.eigh(S)
    Z = V @ np.diag(w ** -0.5) @ V.T  # S^{-1/2}: d = I - Z^T S Z is at rounding level
    Sf = [[Fraction(float(v)) for v in r] for r in S]
    Zf = [[Fraction(float(v)) for v in r] for r in Z]
    for j in (0, 7, 32):
        d = ad.residual_column(S, Z, j, block=5)
        Sz = [sum(Sf[i][k] * Zf[k][j] for k in range(n)) for i in range(n)]
        for i in range(n):
            ex = (1 if i == j else 0) - sum(Zf[k][i] * Sz[k] for k in range(n))
            mag = sum(abs(Zf[k][i]) * sum(abs(Sf[k][l] * Zf[l][j]) for l in range(n)) for k in range(n))
            assert abs(Fraction(float(d[i])) - ex) <= Fraction(U) * abs(ex) + Fraction(U * U) * mag * 40, (i, j)
