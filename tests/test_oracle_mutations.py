"""Planted mistakes in the oracle (CPU only): each mutant must fail a pin.

This shows the pins in test_oracle_pins.py are sharp enough to catch a
dropped term, a wrong sign or a transposed operand anywhere in the oracle."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import sys, os
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import test_oracle_pins as pins


def _paper_stop(err, prev):
    """Algorithm 2's test with reading 2's guards."""
    return err > prev ** 3 or err >= prev or not np.isfinite(err)


def _refine_with(poly_fn=None, update_fn=None, residual_fn=None, stop_fn=None):
    """Algorithm 2 assembled from (possibly mutated) oracle steps, fixed or stopped."""
    poly_fn = poly_fn or oracle.poly
    update_fn = update_fn or oracle.update
    residual_fn = residual_fn or oracle.residual
    stop_fn = stop_fn or _paper_stop

    def refine(S, Z0, m=2, nmax=50, fixed_iters=0):
        if Z0 is None:
            Z0 = oracle.gershgorin_scale(S) * np.eye(S.shape[0])
        Z = np.array(Z0, dtype=np.float64)
        d, err = residual_fn(S, Z)
        hist = [err]
        it = 0
        while it < (fixed_iters or nmax):
            Z = update_fn(Z, poly_fn(d, m))
            prev = err
            d, err = residual_fn(S, Z)
            it += 1
            hist.append(err)
            if not fixed_iters and stop_fn(err, prev):
                break
        return Z, np.array(hist), it
    return refine


def test_unmutated_assembly_passes():
    r = _refine_with()
    pins.check_diagonal(r)
    pins.check_two_by_two(r)
    pins.check_scalar_map(r)
    pins.check_stop_rule(r)


MUTANTS = {
    "dropped_square_term": dict(poly_fn=lambda d, m: 0.5 * d),
    "wrong_sign_linear": dict(poly_fn=lambda d, m: oracle.poly(d, m) - d),
    "wrong_coefficient": dict(poly_fn=lambda d, m: 0.5 * d + 0.25 * oracle.matmul(d, d)),
    "transposed_update": dict(update_fn=lambda Z, Q: Z + oracle.matmul(Q, Z)),
    "residual_sign": dict(residual_fn=lambda S, Z: (lambda r: (-r[0], r[1]))(oracle.residual(S, Z))),
    "residual_missing_transpose": dict(residual_fn=lambda S, Z: (
        lambda X: (np.eye(len(S)) - X, float(np.linalg.norm(np.eye(len(S)) - X))))(
            oracle.matmul(Z, oracle.matmul(S, Z)))),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    r = _refine_with(**MUTANTS[name])
    caught = 0
    for check in (pins.check_diagonal, pins.check_two_by_two, pins.check_scalar_map):
        try:
            check(r)
        except (AssertionError, np.linalg.LinAlgError, FloatingPointError, ValueError):
            caught += 1
    assert caught >= 1, name


STOP_MUTANTS = {
    "square_instead_of_cube": lambda err, prev: err > prev ** 2 or err >= prev or not np.isfinite(err),
    "monotone_guard_dropped": lambda err, prev: err > prev ** 3 or not np.isfinite(err),
    "cube_test_dropped": lambda err, prev: err >= prev or not np.isfinite(err),
}


@pytest.mark.parametrize("name", sorted(STOP_MUTANTS))
def test_stop_mutant_is_caught(name):
    with pytest.raises(AssertionError):
        pins.check_stop_rule(_refine_with(stop_fn=STOP_MUTANTS[name]))


def test_feature_mutants_are_caught():
    def swapped_bounds(S):
        f = oracle.features(S)
        f[2] = 1.0 / f[2] if f[2] else f[2]           # g_hi / g_lo instead of g_lo / g_hi
        return f

    def frobenius_squared(S):
        f = oracle.features(S)
        f[15] = 2.0 * f[15]                           # log ||d0||_F^2 instead of log ||d0||_F
        return f

    def row_sums_signed(S):
        f = oracle.features(S)
        f[5] = np.mean(np.asarray(S).sum(axis=1)) / math.exp(f[1])   # signed instead of absolute sums
        return f

    for bad in (swapped_bounds, frobenius_squared, row_sums_signed):
        with pytest.raises(AssertionError):
            pins.check_features_by_hand(bad)


def test_coefficient_mutants_are_caught(golden):
    def bad1(m):
        c = oracle.coeffs(m)
        c[2] = -c[2]
        return c

    def bad2(m):
        c = oracle.coeffs(m)
        return c[:-1] + [Fraction(0)]

    for bad in (bad1, bad2):
        with pytest.raises(AssertionError):
            pins.check_coefficients(bad, golden)


def test_gradient_mutant_is_caught():
    def bad_backward(P, x, ys, yo, w):
        g = oracle.mlp_backward(P, x, ys, yo, w)
        return g * np.where(np.arange(g.size) % 7 == 0, -1.0, 1.0)

    with pytest.raises(AssertionError):
        pins.check_mlp_gradient(bad_backward)


CONGRUENCE_MUTANTS = {
    "transposed_operand": lambda H, Z: oracle.matmul(Z, oracle.matmul(H, Z.T)),
    "missing_right_factor": lambda H, Z: oracle.matmul(Z.T, H),
    "transpose_dropped": lambda H, Z: oracle.matmul(Z, oracle.matmul(H, Z)),
}


@pytest.mark.parametrize("name", sorted(CONGRUENCE_MUTANTS))
def test_congruence_mutant_is_caught(name):
    bad = CONGRUENCE_MUTANTS[name]
    caught = 0
    for check in (pins.check_congruence_exact, pins.check_congruence_generalized_eigs):
        try:
            check(bad)
        except AssertionError:
            caught += 1
    assert caught >= 1, name
