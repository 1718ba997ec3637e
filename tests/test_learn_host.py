"""Host logic of the learned start's labels (no GPU): the cost model that turns a bulk history into the
modelled time of a whole factorization, and the least-squares fit that calibrates it."""
import math

import numpy as np
import pytest

from paper_2404_19163_gb300 import learn

# a model with round constants: iteration 1 ms + 1e-12 N^3 s, residual 2 ms + 2e-12 N^3, update 3 ms + 3e-12 N^3
MODEL = {"iter": {q: (0.001, 1e-12) for q in (2, 3, 4, 5)}, "res": (0.002, 2e-12), "upd": (0.003, 3e-12),
         "source": "test"}


def test_work_is_bulk_plus_refinement():
    # N = 1000: an iteration 2 ms, a residual 4 ms, an update 6 ms.  Three bulk updates end at
    # Err = 1e-5; the refinement's order 2 gives 1e-15 / 1000 < tol sqrt(N) / 2, so one update and
    # two residuals (before and after it).
    t = learn.work([0.5, 0.1, 1e-3, 1e-5], 1000, 2, 1e-4, model=MODEL)
    assert t == pytest.approx(3 * 0.002 + 2 * 0.004 + 1 * 0.006)


def test_work_counts_a_second_update_when_one_cannot_reach_tol():
    # Err = 0.3 at N = 1000: no order up to 5 brings 0.3^(m+1) / N^(m/2) to half the target, so the
    # first update takes the bulk's order (2): 0.027 / 1000 = 2.7e-5, then a second update (order 2)
    # reaches it.  One bulk update, three residuals, two updates.
    t = learn.work([0.9, 0.3], 1000, 2, 1.0, model=MODEL)
    assert t == pytest.approx(1 * 0.002 + 3 * 0.004 + 2 * 0.006)


def test_work_is_infinite_for_failed_bulks():
    assert learn.work([0.5, float("nan")], 1000, 2, 1.0, model=MODEL) == math.inf
    assert learn.work([], 1000, 2, 1.0, model=MODEL) == math.inf
    # a bulk that never got below tau (per sqrt(N))
    assert learn.work([0.5, 0.2], 100, 2, 1e-3, model=MODEL) == math.inf


def test_fit_recovers_a_plus_b_n_cubed():
    ns = np.array([128, 512, 1024, 4096], dtype=np.float64)
    ts = 2e-4 + 3e-13 * ns ** 3
    a, b = learn._fit(ns, ts)
    assert a == pytest.approx(2e-4, rel=1e-9) and b == pytest.approx(3e-13, rel=1e-9)
