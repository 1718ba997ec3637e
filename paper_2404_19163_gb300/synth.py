"""Seeded synthetic overlap matrices (inputs only; none of the method's arithmetic).

Shared by the tests, the benchmark and the CPU oracle's drivers.  Every matrix
is FP64, row-major, symmetric positive definite.  Seeds follow
``numpy.random.default_rng(20240429 + 1000 * workload + k)``.

Workloads (the paper's real Ag561 overlap matrix, Sec. 5.4, is not available;
the Gaussian-overlap models below stand in for it):

* ``householder_spd``   S = Q diag(lam) Q^T, Q a product of N Householder
                        reflections, lam log-uniform in [0.2, 5] (cond ~ 25).
* ``cubic_overlap``     s-type Gaussians exp(-r^2/2) on a jittered cubic
                        lattice (16^3 sites, spacing 2.5, jitter 0.1): N = 4096.
* ``fcc_overlap``       normalised s-Gaussians with 4 exponents per site on an
                        fcc lattice; the lattice constant sets cond ~ 1e5-1e6.
* ``cluster_overlap``   random cluster geometries (points in a sphere at the
                        cubic-lattice density, minimum distance 1.5) for the
                        batched trajectory workload.
* ``paper_synthetic``   Sec. 5.1's test matrix exp(-|i-j|/2) sin(i+1),
                        symmetrised and shifted so lambda_min = gamma.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 20240429


def rng(workload: int, k: int = 0) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + 1000 * workload + k)


# ------------------------------------------------------------------ workload 1
def householder_spd(n: int = 256, seed: int = 0, lam_lo: float = 0.2, lam_hi: float = 5.0):
    """S = Q diag(lam) Q^T with Q = H_1 ... H_n (Householder, v ~ N(0,1)).
    Returns (S, Q, lam)."""
    g = rng(1, seed)
    Q = np.eye(n)
    for _ in range(n):
        v = g.standard_normal(n)
        v /= np.linalg.norm(v)
        Q -= 2.0 * np.outer(Q @ v, v)
    lam = np.exp(g.uniform(math.log(lam_lo), math.log(lam_hi), n))
    S = (Q * lam) @ Q.T
    S = 0.5 * (S + S.T)
    return S, Q, lam


# ------------------------------------------------------------------ Gaussian overlaps
def gaussian_overlap(pos, exps=None, out=None, chunk: int = 1024):
    """S_ij = (2 sqrt(a_i a_j) / (a_i + a_j))^{3/2} exp(-a_i a_j / (a_i + a_j) r_ij^2),
    the overlap of two normalised s-type Gaussians; with all a = 1 this is
    exp(-r_ij^2 / 2).  ``pos`` (n, 3) holds one centre per basis function."""
    pos = np.asarray(pos, dtype=np.float64)
    n = pos.shape[0]
    a = np.ones(n) if exps is None else np.asarray(exps, dtype=np.float64)
    S = np.empty((n, n)) if out is None else out
    sq = np.sum(pos * pos, axis=1)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        r2 = sq[r0:r1, None] + sq[None, :] - 2.0 * pos[r0:r1] @ pos.T
        np.maximum(r2, 0.0, out=r2)
        ai = a[r0:r1, None]
        asum = ai + a[None, :]
        pref = (2.0 * np.sqrt(ai * a[None, :]) / asum) ** 1.5
        S[r0:r1] = pref * np.exp(-(ai * a[None, :] / asum) * r2)
    # exact symmetry and unit diagonal (normalised functions)
    S[...] = 0.5 * (S + S.T)
    np.fill_diagonal(S, 1.0)
    return S


def cubic_sites(n_side: int = 16, spacing: float = 2.5, jitter: float = 0.1, seed: int = 0,
                workload: int = 2):
    g = rng(workload, seed)
    ax = np.arange(n_side) * spacing
    pos = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1).reshape(-1, 3)
    return pos + g.normal(0.0, jitter, pos.shape)


def cubic_overlap(n_side: int = 16, spacing: float = 2.5, jitter: float = 0.1, seed: int = 0):
    """Workload 2: 16^3 = 4096 s-type sites, S_ij = exp(-r^2/2), unit diagonal."""
    return gaussian_overlap(cubic_sites(n_side, spacing, jitter, seed))


FCC_EXPONENTS = (0.3, 0.3 * (5.0 ** (1.0 / 3.0)), 0.3 * (5.0 ** (2.0 / 3.0)), 1.5)  # geometric in [0.3, 1.5]
FCC_LATTICE = 3.6


def fcc_sites(cells=(8, 8, 16), a_lat: float = FCC_LATTICE, jitter: float = 0.0, seed: int = 0,
              workload: int = 3):
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    cx, cy, cz = cells
    grid = np.stack(np.meshgrid(np.arange(cx), np.arange(cy), np.arange(cz), indexing="ij"),
                    axis=-1).reshape(-1, 3)
    pos = ((grid[:, None, :] + basis[None, :, :]).reshape(-1, 3)) * a_lat
    if jitter > 0:
        pos = pos + rng(workload, seed).normal(0.0, jitter, pos.shape)
    return pos


def fcc_basis(pos, exps=FCC_EXPONENTS):
    """Centres and exponents of the basis: every site carries every exponent."""
    k = len(exps)
    centres = np.repeat(pos, k, axis=0)
    a = np.tile(np.asarray(exps, dtype=np.float64), pos.shape[0])
    return centres, a


def fcc_overlap(cells=(8, 8, 16), a_lat: float = FCC_LATTICE, exps=FCC_EXPONENTS,
                jitter: float = 0.0, seed: int = 0, perturb: float = 0.0, perturb_seed: int = 1):
    """Workload 3: fcc sites (4 per cell) x 4 exponents; (8, 8, 16) cells give
    N = 16384.  ``perturb`` > 0 displaces every site by N(0, perturb^2)
    (the neighbouring geometry whose converged Z warm-starts this one)."""
    pos = fcc_sites(cells, a_lat, jitter, seed)
    if perturb > 0:
        pos = pos + rng(3, 100 + perturb_seed).normal(0.0, perturb, pos.shape)
    c, a = fcc_basis(pos, exps)
    return gaussian_overlap(c, a)


# ------------------------------------------------------------------ workload 4: trajectories
CUBIC_DENSITY = 1.0 / 2.5 ** 3


def cluster_sites(n: int, seed: int, min_dist: float = 1.5, density: float = CUBIC_DENSITY,
                  workload: int = 4):
    """n random points in a sphere of volume n/density, no two closer than min_dist
    (random sequential addition; candidates are tested in batches against a KD-tree)."""
    from scipy.spatial import cKDTree
    g = rng(workload, seed)
    radius = (3.0 * n / (4.0 * math.pi * density)) ** (1.0 / 3.0)
    pts = np.empty((0, 3))
    while pts.shape[0] < n:
        cand = g.uniform(-radius, radius, (2 * n, 3))
        cand = cand[np.sum(cand * cand, axis=1) <= radius * radius]
        if pts.shape[0]:
            d, _ = cKDTree(pts).query(cand, k=1)
            cand = cand[d >= min_dist]
        # within the batch, keep the first of every conflicting pair (sequential order)
        keep = np.ones(cand.shape[0], dtype=bool)
        for a, b in sorted(cKDTree(cand).query_pairs(min_dist)):
            if keep[a] and keep[b]:
                keep[b] = False
        cand = cand[keep]
        pts = np.vstack([pts, cand[: n - pts.shape[0]]])
    return pts


def gaussian_overlap_torch(pos, exps=None, device="cuda", chunk: int = 4096):
    """The overlap of ``gaussian_overlap`` built on a torch device (FP64), row chunk by chunk."""
    import torch
    p = torch.as_tensor(np.asarray(pos, dtype=np.float64), device=device)
    n = p.shape[0]
    a = torch.ones(n, dtype=torch.float64, device=device) if exps is None else \
        torch.as_tensor(np.asarray(exps, dtype=np.float64), device=device)
    sq = (p * p).sum(dim=1)
    S = torch.empty((n, n), dtype=torch.float64, device=device)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        r2 = (sq[r0:r1, None] + sq[None, :] - 2.0 * (p[r0:r1] @ p.T)).clamp_min_(0.0)
        ai = a[r0:r1, None]
        asum = ai + a[None, :]
        pref = (2.0 * torch.sqrt(ai * a[None, :]) / asum) ** 1.5
        S[r0:r1] = pref * torch.exp(-(ai * a[None, :] / asum) * r2)
    S = 0.5 * (S + S.T)
    S.fill_diagonal_(1.0)
    return S.contiguous()


def fcc_overlap_torch(cells=(8, 8, 16), a_lat: float = FCC_LATTICE, exps=FCC_EXPONENTS, perturb: float = 0.0,
                      perturb_seed: int = 1, device="cuda"):
    """``fcc_overlap`` built on a torch device."""
    pos = fcc_sites(cells, a_lat)
    if perturb > 0:
        pos = pos + rng(3, 100 + perturb_seed).normal(0.0, perturb, pos.shape)
    c, a = fcc_basis(pos, exps)
    return gaussian_overlap_torch(c, a, device=device)


def trajectory(count: int = 128, n_lo: int = 256, n_hi: int = 3072, frames: int = 11,
               sigma: float = 0.02, seed: int = 0):
    """Workload 4: ``count`` independent clusters with N_i ~ U[n_lo, n_hi];
    frame f displaces every site by N(0, sigma^2) from frame f-1.
    Returns (sizes, frame_fn) where frame_fn(f) -> list of S matrices."""
    g = rng(4, 10_000 + seed)
    sizes = g.integers(n_lo, n_hi + 1, count)
    base = [cluster_sites(int(n), seed * 100_000 + i) for i, n in enumerate(sizes)]

    def positions(f):
        out = []
        for i, p in enumerate(base):
            q = p.copy()
            gi = rng(4, 20_000 + seed * 1000 + i)
            for _ in range(f):
                q = q + gi.normal(0.0, sigma, q.shape)
            out.append(q)
        return out

    def frame(f):
        return [gaussian_overlap(p) for p in positions(f)]

    frame.positions = positions
    return sizes, frame


# ------------------------------------------------------------------ workload 5: proposal data
def proposal_sites(k: int, n_lo: int = 128, n_hi: int = 4096, split: str = "train"):
    """Geometry of one training/held-out overlap matrix for the start-proposal network:
    (centres (n, 3), exponents (n,) or None for unit exponents).  N is log-uniform in
    [n_lo, n_hi]; the conditioning is varied through the lattice spacing and the exponent
    range (Gaussian-overlap models, cond roughly 10 ... 1e6)."""
    g = rng(5, (0 if split == "train" else 1_000_000) + k)
    n_target = int(round(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
    kind = g.integers(0, 3)
    # the spacing ranges spread cond(S) over 10 ... 1e6 (measured with eigvalsh on samples of each kind
    # up to N = 1800: cluster and cubic blocks ~10 ... 2e4, fcc blocks ~40 ... 1e6; cond grows with N)
    if kind == 0:      # single exponent, random cluster, spacing sets the conditioning
        d = g.uniform(1.0, 1.6)
        return cluster_sites(n_target, int(g.integers(1 << 30)), min_dist=0.8 * d, density=1.0 / d ** 3,
                             workload=5), None
    if kind == 1:      # jittered cubic block
        side = max(2, int(round(n_target ** (1.0 / 3.0))))
        return cubic_sites(side, g.uniform(1.0, 1.75), 0.1, int(g.integers(1 << 30)), workload=5), None
    # multi-exponent fcc block (ill-conditioned end)
    # (exponents in a geometric sequence from 0.3 with ratio 1.5 ... 2.5: closer ratios make the functions
    # of one site nearly parallel and cond(S) leaves the range)
    nexp = int(g.integers(2, 5))
    exps = 0.3 * g.uniform(1.5, 2.5) ** np.arange(nexp)
    cells_total = max(1, n_target // (4 * nexp))
    cz = max(1, int(round(cells_total ** (1.0 / 3.0))))
    cells = (cz, cz, max(1, cells_total // (cz * cz)))
    pos = fcc_sites(cells, g.uniform(3.0, 6.0), 0.05, int(g.integers(1 << 30)), workload=5)
    return fcc_basis(pos, exps)


def proposal_instance(k: int, n_lo: int = 128, n_hi: int = 4096, split: str = "train"):
    """S of ``proposal_sites`` built on the host (NumPy)."""
    pos, exps = proposal_sites(k, n_lo, n_hi, split)
    return gaussian_overlap(pos, exps)


def proposal_instance_torch(k: int, n_lo: int = 128, n_hi: int = 4096, split: str = "train", device="cuda"):
    """S of ``proposal_sites`` built on a torch device (the same matrix up to rounding)."""
    pos, exps = proposal_sites(k, n_lo, n_hi, split)
    return gaussian_overlap_torch(pos, exps, device=device)


# ------------------------------------------------------------------ the paper's own test matrix
def paper_synthetic(n: int, gamma: float = 0.5):
    """Sec. 5.1: T_ij = exp(-|i-j|/2) sin(i+1) (1-based i), symmetrised as
    (T + T^T)/2 (T itself is not symmetric), then shifted by (gamma - lambda_min) I."""
    i = np.arange(1, n + 1, dtype=np.float64)
    T = np.exp(-np.abs(i[:, None] - i[None, :]) / 2.0) * np.sin(i + 1.0)[:, None]
    S = 0.5 * (T + T.T)
    lmin = float(np.linalg.eigvalsh(S)[0])
    S[np.diag_indices(n)] += gamma - lmin
    return S


def paper_synthetic_torch(n: int, gamma: float = 0.5, device="cuda"):
    """``paper_synthetic`` built on a torch device (FP64; lambda_min from torch.linalg.eigvalsh)."""
    import torch
    i = torch.arange(1, n + 1, dtype=torch.float64, device=device)
    T = torch.exp(-(i[:, None] - i[None, :]).abs() / 2.0) * torch.sin(i + 1.0)[:, None]
    S = 0.5 * (T + T.T)
    del T
    lmin = float(torch.linalg.eigvalsh(S)[0])
    S.diagonal().add_(gamma - lmin)
    return S.contiguous()


def paper_start_torch(S, alpha: float = 0.005, seed: int = 0, chunk: int = 2048):
    """Sec. 5.1's start Z0 = S^{-1/2} + alpha U, U_ij ~ U(-0.5, 0.5), on S's device.  S^{-1/2} is
    V diag(lambda^{-1/2}) V^T from torch.linalg.eigh (the paper builds it with cuSOLVER too)."""
    import torch
    lam, V = torch.linalg.eigh(S)
    Z0 = (V * lam.rsqrt()) @ V.T
    del V
    n = S.shape[0]
    g = rng(6, seed)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        Z0[r0:r1] += torch.as_tensor(alpha * g.uniform(-0.5, 0.5, (r1 - r0, n)), device=S.device)
    return Z0.contiguous()


def random_warm_start(n: int, alpha: float, seed: int = 0, workload: int = 6):
    """alpha * U with U_ij ~ U(-0.5, 0.5) (Sec. 5.1's perturbation of S^{-1/2})."""
    return alpha * rng(workload, seed).uniform(-0.5, 0.5, (n, n))
