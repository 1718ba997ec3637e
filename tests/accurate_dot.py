"""Residual columns d_j = e_j - Z^T S z_j in about twice FP64 precision (test infrastructure).

Built from error-free transformations: Knuth's TwoSum (a + b = s + e exactly) and Dekker's
TwoProduct through Veltkamp splitting (a b = p + e exactly, no FMA needed), with the products
of a row summed by a pairwise cascade whose rounding errors are collected and added back, in the
spirit of Ogita, Rump and Oishi, "Accurate sum and dot product" (SIAM J. Sci. Comput., 2005).
A sum of n products comes out as an unevaluated pair hi + lo with error about
u^2 (log2 n + 2) sum|a_k b_k| + u^2 |sum|, u = 2^-53: far below the FP64 rounding of the
result, so it serves as the exact value when judging an FP64-accurate residual.

Each step is a separate element-wise operation, so the same code runs on numpy arrays and on
torch tensors (CPU or CUDA) without any fused multiply-add that would spoil the exactness.
"""
import numpy as np

_SPLITTER = 134217729.0  # 2^27 + 1


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def two_sum(a, b):
    s = a + b
    z = s - a
    return s, (a - (s - z)) + (b - z)


def split(a):
    c = _SPLITTER * a
    h = c - (c - a)
    return h, a - h


def two_prod(a, b):
    p = a * b
    ah, al = split(a)
    bh, bl = split(b)
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def row_sums_dd(P):
    """Row sums of the 2-D array P as (hi, lo), hi + lo ~ the exact sums."""
    P = P.clone() if _is_torch(P) else P.copy()
    err = P[:, 0] * 0.0
    while P.shape[1] > 1:
        m = P.shape[1]
        if m % 2:
            s, e = two_sum(P[:, 0], P[:, m - 1])
            P[:, 0] = s
            err = err + e
            P = P[:, : m - 1]
            m -= 1
        s, e = two_sum(P[:, 0:m:2], P[:, 1:m:2])
        err = err + e.sum(1)
        P = s
    return two_sum(P[:, 0], err)


def matvec_dd(A, x_hi, x_lo=None, block=2048):
    """A (x_hi + x_lo) row by row as (hi, lo).  A may be a strided view (e.g. a transpose)."""
    n = A.shape[0]
    his, los = [], []
    for r0 in range(0, n, block):
        Ab = A[r0:r0 + block]
        p, e = two_prod(Ab, x_hi[None, :])
        hi, lo = row_sums_dd(p)
        lo = lo + e.sum(1)
        if x_lo is not None:
            lo = lo + (Ab * x_lo[None, :]).sum(1)
        hi, lo = two_sum(hi, lo)
        his.append(hi)
        los.append(lo)
    if _is_torch(A):
        import torch
        return torch.cat(his), torch.cat(los)
    return np.concatenate(his), np.concatenate(los)


def residual_column(S, Z, j, block=2048):
    """Column j of d = I - Z^T S Z (S symmetric), rounded once to FP64 from the accurate value."""
    v_hi, v_lo = matvec_dd(S, Z[:, j], block=block)          # S z_j (rows of S = its columns)
    w_hi, w_lo = matvec_dd(Z.T, v_hi, v_lo, block=block)     # Z^T (S z_j)
    d = -w_hi
    d[j] = d[j] + 1.0  # exact: w_hi[j] is within a factor 2 of 1 whenever d is small
    return d - w_lo
