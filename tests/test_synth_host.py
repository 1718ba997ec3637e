"""The seeded input recipes (no GPU): each generator gives the structure its workload states, and the same
seed gives the same matrix.  Small sizes, so the checks stay cheap."""
import math

import numpy as np

from paper_2404_19163_gb300 import synth


def test_householder_spd_spectrum_and_seed():
    S, Q, lam = synth.householder_spd(64, seed=3)
    assert np.allclose(S, S.T, atol=0)
    assert np.allclose(Q.T @ Q, np.eye(64), atol=1e-12)
    ev = np.linalg.eigvalsh(S)
    assert 0.2 * (1 - 1e-10) <= ev[0] and ev[-1] <= 5.0 * (1 + 1e-10)
    assert np.allclose(np.sort(lam), ev, rtol=1e-10)
    S2, _, _ = synth.householder_spd(64, seed=3)
    assert np.array_equal(S, S2)
    S3, _, _ = synth.householder_spd(64, seed=4)
    assert not np.array_equal(S, S3)


def test_cubic_overlap_is_a_unit_diagonal_spd_overlap():
    S = synth.cubic_overlap(n_side=6)
    assert S.shape == (216, 216)
    assert np.array_equal(S, S.T)
    assert np.allclose(np.diag(S), 1.0)
    assert np.all(S > 0) and np.all(S <= 1.0)
    ev = np.linalg.eigvalsh(S)
    # spacing 2.5 with small jitter: well conditioned, as measured on the full 16^3 lattice (cond ~ 1.7)
    assert ev[0] > 0.5 and ev[-1] / ev[0] < 3.0
    assert np.array_equal(S, synth.cubic_overlap(n_side=6))


def test_trajectory_sizes_and_small_frame_steps():
    sizes, frame = synth.trajectory(count=6, n_lo=40, n_hi=90, frames=3)
    assert len(sizes) == 6 and all(40 <= int(n) <= 90 for n in sizes)
    p0, p1 = frame.positions(0), frame.positions(1)
    for a, b, n in zip(p0, p1, sizes):
        assert a.shape == (int(n), 3)
        d = np.abs(b - a)
        assert 0 < d.max() < 0.2  # N(0, 0.02^2) per coordinate per frame
    S = frame(1)
    for s, n in zip(S, sizes):
        assert s.shape == (int(n), int(n)) and np.allclose(np.diag(s), 1.0)
        assert np.linalg.eigvalsh(s)[0] > 0


def test_paper_synthetic_is_shifted_to_gamma():
    S = synth.paper_synthetic(200, gamma=0.5)
    assert np.array_equal(S, S.T)
    ev = np.linalg.eigvalsh(S)
    assert abs(ev[0] - 0.5) < 1e-12
    # the unshifted matrix is T's symmetric part: off-diagonal entries unchanged by the shift
    i = np.arange(1, 201, dtype=np.float64)
    T = np.exp(-np.abs(i[:, None] - i[None, :]) / 2.0) * np.sin(i + 1.0)[:, None]
    off = ~np.eye(200, dtype=bool)
    assert np.allclose(S[off], (0.5 * (T + T.T))[off], atol=0)


def test_proposal_instances_span_sizes_and_are_spd():
    ns = []
    for k in range(6):
        S = synth.proposal_instance(k, n_lo=64, n_hi=256)
        n = S.shape[0]
        ns.append(n)
        assert 64 <= n <= 256 and np.allclose(S, S.T)
        assert np.linalg.eigvalsh(S)[0] > 0
    assert len(set(ns)) > 1
    # train and held-out draws differ
    assert not np.array_equal(synth.proposal_instance(0, 64, 256, "train"),
                              synth.proposal_instance(0, 64, 256, "heldout"))
