"""Plain CPU oracle for the inverse-overlap factorization Z Z^T = S^{-1}.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2404_19163_gb300``) never imports it, and
the two share no code: the only common dependency is the seeded input
generator module, which holds none of the method's arithmetic.

Contents, each following arXiv:2404.19163 (Habib, Finkelstein, Niklasson):

* ``refine``            Algorithm 2 (parameter-free stop) / Algorithm 1
                        (tolerance stop) in FP64, delta-form of Eq. np1;
                        the dense loops are plain C (``zfact_oracle.c``).
* ``refine_alg3``       Algorithm 3: the stop of Algorithm 2 followed by the
                        refinement update(s).
* ``congruence``        H_perp = Z^T H Z (Sec. 2, Eq. standard_form), the transform
                        the factor exists for.
* ``coeffs``            c_k = binom(2k,k)/4^k, exact rationals (Sec. 3; the
                        m = 2 case equals Appendix A's a_k after X = I - d).
* ``split16``           Eq. splitStyle: A^(h) = FP16[A], A^(l) = FP16[A - FP32[A^(h)]]
                        (and the same with BF16), with an optional power-of-two
                        scale applied first.
* ``round16``           FP16 / BF16 rounding of FP32 values (round to nearest even).
* ``mm16``              a product of 16-bit-rounded operands evaluated in FP64
                        (the exact value a tensor-core product approximates).
* ``scalar_map_hist``   the residual history predicted by the scalar map
                        g(x) = x p(1-x)^2 applied to the spectrum of X0.
* ``features``          the 16 start-proposal features of an overlap matrix.
* ``mlp_*``             forward / backward / Adam of the start-proposal MLP in FP64.

Parity unpinned: none of the functions above; every one has a pin in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "zfact_oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (gcc, OpenMP) into oracle/_build."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.zo_matmul.argtypes = [P, P, P, I64]
        lib.zo_atb_sym.argtypes = [P, P, P, I64]
        lib.zo_residual.argtypes = [P, P, P, I64]
        lib.zo_congruence.argtypes = [P, P, P, I64]
        lib.zo_residual.restype = ctypes.c_double
        lib.zo_poly.argtypes = [P, ctypes.c_int, P, I64]
        lib.zo_update.argtypes = [P, P, I64]
        lib.zo_gershgorin_scale.argtypes = [P, I64]
        lib.zo_gershgorin_scale.restype = ctypes.c_double
        lib.zo_coeffs.argtypes = [ctypes.c_int, P]
        lib.zo_refine.argtypes = [P, P, I64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_double, P, P, ctypes.c_int]
        lib.zo_refine.restype = ctypes.c_int
        lib.zo_num_threads.restype = ctypes.c_int
        lib.zo_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data


def num_threads() -> int:
    return _load().zo_num_threads()


def set_threads(t: int) -> None:
    _load().zo_set_threads(int(t))


# ---------------------------------------------------------------- dense FP64 steps
def matmul(A, B):
    """C = A B in FP64 (plain triple loop)."""
    A, pa = _c(A)
    B, pb = _c(B)
    n = A.shape[0]
    C = np.empty((n, n))
    _load().zo_matmul(pa, pb, C.ctypes.data, n)
    return C


def residual(S, Z):
    """d = I - Z^T S Z (upper triangle mirrored) and ||d||_F (Eq. np1, Algorithm 2)."""
    S, ps = _c(S)
    Z, pz = _c(Z)
    n = S.shape[0]
    d = np.empty((n, n))
    err = _load().zo_residual(ps, pz, d.ctypes.data, n)
    return d, err


def congruence(H, Z):
    """H_perp = Z^T H Z, upper triangle mirrored (Sec. 2, Eq. standard_form)."""
    H, ph = _c(H)
    Z, pz = _c(Z)
    n = H.shape[0]
    Hp = np.empty((n, n))
    _load().zo_congruence(ph, pz, Hp.ctypes.data, n)
    return Hp


def poly(d, m):
    """Q = p_m(d) - I = sum_{k=1..m} c_k d^k."""
    d, pd = _c(d)
    n = d.shape[0]
    Q = np.empty((n, n))
    _load().zo_poly(pd, int(m), Q.ctypes.data, n)
    return Q


def update(Z, Q):
    """Z + Z Q (Z_{n+1} = Z_n p(d_n))."""
    Z = np.array(Z, dtype=np.float64, copy=True, order="C")
    Q, pq = _c(Q)
    _load().zo_update(Z.ctypes.data, pq, Z.shape[0])
    return Z


def gershgorin_scale(S) -> float:
    """1/sqrt(max_i sum_j |S_ij|): Z0 = s I gives ||X0 - I||_2 < 1 for SPD S."""
    S, ps = _c(S)
    return _load().zo_gershgorin_scale(ps, S.shape[0])


def refine(S, Z0=None, m=2, nmax=50, fixed_iters=0, rule=0, tol=0.0):
    """Algorithm 2 (rule 0) or Algorithm 1 (rule 1) in FP64.

    Returns (Z, hist, iters): hist[0] = ||I - Z0^T S Z0||_F and hist[i] the
    Err of the i-th update.  iters < 0 signals a non-finite Err."""
    S, ps = _c(S)
    n = S.shape[0]
    if Z0 is not None:
        Z0, pz0 = _c(Z0)
    else:
        pz0 = None
    Z = np.empty((n, n))
    cap = max(nmax, fixed_iters) + 1
    hist = np.full(cap, np.nan)
    it = _load().zo_refine(ps, pz0, n, int(m), int(nmax), int(fixed_iters), int(rule),
                           float(tol), Z.ctypes.data, hist.ctypes.data, cap)
    used = (it if it >= 0 else int(np.sum(np.isfinite(hist)))) + 1
    return Z, hist[:max(used, 1)], it


def refine_alg3(S, Z0=None, m=2, nmax=50, refine_steps=1):
    """Algorithm 3: Algorithm 2, then ``refine_steps`` further updates
    (the oracle is FP64 throughout, so the precision change of Algorithm 3 is
    the identity here), then the residual of the returned Z.
    Returns (Z, hist, iters) with hist extended by the refinement residuals."""
    Z, hist, it = refine(S, Z0, m=m, nmax=nmax)
    hist = list(hist)
    for _ in range(refine_steps):
        d, _ = residual(S, Z)
        Z = update(Z, poly(d, m))
        hist.append(residual(S, Z)[1])
    return Z, np.array(hist), it


# ---------------------------------------------------------------- coefficients
def coeffs(m: int):
    """Exact c_k = binom(2k,k)/4^k for k = 0..m (Taylor series of (1-t)^{-1/2})."""
    return [Fraction(math.comb(2 * k, k), 4 ** k) for k in range(m + 1)]


# ---------------------------------------------------------------- 16-bit formats
def round16(a32, kind: str):
    """Round FP32 values to FP16 or BF16 (round to nearest, ties to even),
    returned as float32 arrays holding the 16-bit values."""
    a32 = np.asarray(a32, dtype=np.float32)
    if kind == "fp16":
        return a32.astype(np.float16).astype(np.float32)
    if kind == "bf16":
        import torch
        return torch.from_numpy(np.ascontiguousarray(a32)).to(torch.bfloat16).to(torch.float32).numpy()
    raise ValueError(kind)


def split16(A, kind: str = "fp16", scale: float = 1.0):
    """Eq. splitStyle (Sec. 3.1): with A32 = FP32[scale * A],
    hi = R16[A32] and lo = R16[A32 - FP32[hi]], R16 the FP16 (or BF16) rounding.
    ``scale`` is a power of two, so it changes no significand bits.
    Returns (hi, lo) as float32 arrays holding 16-bit values."""
    a32 = (np.asarray(A, dtype=np.float64) * scale).astype(np.float32)
    hi = round16(a32, kind)
    lo = round16(a32 - hi, kind)
    return hi, lo


def mm16(A16, B16):
    """Product of operands already rounded to 16 bits, in FP64: the value a
    tensor-core product with FP32 accumulation approximates."""
    return np.asarray(A16, np.float64) @ np.asarray(B16, np.float64)


# ---------------------------------------------------------------- scalar map
def scalar_map_hist(mu, m: int, n_iters: int, dps: int = 50):
    """Residual history predicted from the spectrum mu of X0 alone.

    X_{n+1} = p(d_n)^T X_n p(d_n) with p a polynomial in X_n, so every
    eigenvalue evolves by g(x) = x p_m(1 - x)^2 independently, whatever Z0
    is; then ||X_n - I||_F = sqrt(sum_i (1 - g^n(mu_i))^2).  Evaluated in
    mpmath at ``dps`` digits."""
    import mpmath as mp
    mp.mp.dps = dps
    c = [mp.mpf(f.numerator) / f.denominator for f in coeffs(m)]
    xs = [mp.mpf(float(x)) for x in np.asarray(mu, dtype=np.float64).ravel()]
    out = []
    for it in range(n_iters + 1):
        out.append(float(mp.sqrt(mp.fsum((1 - x) ** 2 for x in xs))))
        nxt = []
        for x in xs:
            t = 1 - x
            p = mp.fsum(c[k] * t ** k for k in range(m + 1))
            nxt.append(x * p * p)
        xs = nxt
    return np.array(out)


# ---------------------------------------------------------------- start-proposal features
N_FEATURES = 16


def features(S):
    """The 16 start-proposal features of an overlap matrix S (FP64).

    With Gershgorin bounds g_hi = max_i (S_ii + sum_{j!=i} |S_ij|),
    g_lo = min_i (S_ii - sum_{j!=i} |S_ij|), s0 = 1/sqrt(g_hi), X0 = s0^2 S,
    d0 = I - X0 and moments t_k = tr(d0^k)/N (k = 1..4):
      0 log N, 1 log g_hi, 2 g_lo/g_hi, 3 mean S_ii/g_hi, 4 min S_ii/g_hi,
      5 mean row |S| sum / g_hi, 6 min row |S| sum / g_hi,
      7..10 t_1..t_4, 11 sqrt(t_2), 12 t_2 - t_1^2,
      13 t_3 - 3 t_1 t_2 + 2 t_1^3, 14 t_4 - 4 t_1 t_3 + 6 t_1^2 t_2 - 3 t_1^4,
      15 log ||d0||_F."""
    S = np.asarray(S, dtype=np.float64)
    n = S.shape[0]
    diag = np.diag(S).copy()
    rows = np.abs(S).sum(axis=1)
    off = rows - np.abs(diag)
    g_hi = float(np.max(diag + off))
    g_lo = float(np.min(diag - off))
    s2 = 1.0 / g_hi
    d0 = -s2 * S
    d0[np.diag_indices(n)] += 1.0
    d2 = matmul(d0, d0)
    t1 = float(np.trace(d0)) / n
    t2 = float(np.sum(d0 * d0)) / n
    t3 = float(np.sum(d2 * d0)) / n
    t4 = float(np.sum(d2 * d2)) / n
    f = np.array([
        math.log(n), math.log(g_hi), g_lo / g_hi, diag.mean() / g_hi, diag.min() / g_hi,
        rows.mean() / g_hi, rows.min() / g_hi, t1, t2, t3, t4, math.sqrt(t2), t2 - t1 * t1,
        t3 - 3 * t1 * t2 + 2 * t1 ** 3, t4 - 4 * t1 * t3 + 6 * t1 * t1 * t2 - 3 * t1 ** 4,
        math.log(math.sqrt(t2 * n)),
    ])
    return f


# ---------------------------------------------------------------- start-proposal MLP (FP64)
MLP_SIZES = (16, 64, 64, 5)   # inputs, hidden, hidden, outputs (log-scale, 4 order logits)
ORDERS = (2, 3, 4, 5)


def gelu(x):
    """GELU(x) = x Phi(x), Phi the standard normal CDF."""
    from scipy.special import erf
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def mlp_unpack(params):
    """Flat parameter vector -> [(W1, b1), (W2, b2), (W3, b3)], W_l of shape (out, in)."""
    params = np.asarray(params, dtype=np.float64)
    out, off = [], 0
    for fi, fo in zip(MLP_SIZES[:-1], MLP_SIZES[1:]):
        W = params[off:off + fo * fi].reshape(fo, fi)
        off += fo * fi
        b = params[off:off + fo]
        off += fo
        out.append((W, b))
    assert off == params.size
    return out


def mlp_num_params():
    return sum(fo * fi + fo for fi, fo in zip(MLP_SIZES[:-1], MLP_SIZES[1:]))


def mlp_forward(params, x):
    """y = W3 gelu(W2 gelu(W1 x + b1) + b2) + b3 for a batch x of shape (B, 16)."""
    (W1, b1), (W2, b2), (W3, b3) = mlp_unpack(params)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    return h2 @ W3.T + b3


def mlp_loss(params, x, y_scale, y_order, w_order=1.0):
    """Mean over the batch of (y0 - t)^2 + w * CE(softmax(y1..4), order)."""
    y = mlp_forward(params, x)
    B = y.shape[0]
    r = y[:, 0] - y_scale
    lg = y[:, 1:]
    mx = lg.max(axis=1, keepdims=True)
    lse = (mx[:, 0] + np.log(np.exp(lg - mx).sum(axis=1)))
    ce = lse - lg[np.arange(B), y_order]
    return float(np.mean(r * r + w_order * ce))


def mlp_backward(params, x, y_scale, y_order, w_order=1.0):
    """Gradient of ``mlp_loss`` with respect to the flat parameter vector
    (reverse-mode chain rule written out layer by layer)."""
    (W1, b1), (W2, b2), (W3, b3) = mlp_unpack(params)
    x = np.asarray(x, dtype=np.float64)
    B = x.shape[0]
    z1 = x @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    y = h2 @ W3.T + b3
    gy = np.zeros_like(y)
    gy[:, 0] = 2.0 * (y[:, 0] - y_scale) / B
    lg = y[:, 1:]
    e = np.exp(lg - lg.max(axis=1, keepdims=True))
    sm = e / e.sum(axis=1, keepdims=True)
    sm[np.arange(B), y_order] -= 1.0
    gy[:, 1:] = w_order * sm / B
    gW3 = gy.T @ h2
    gb3 = gy.sum(axis=0)
    gh2 = gy @ W3
    gz2 = gh2 * gelu_grad(z2)
    gW2 = gz2.T @ h1
    gb2 = gz2.sum(axis=0)
    gh1 = gz2 @ W2
    gz1 = gh1 * gelu_grad(z1)
    gW1 = gz1.T @ x
    gb1 = gz1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def adam_step(params, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1); t is the 1-based step."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
