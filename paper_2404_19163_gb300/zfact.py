"""Thin ctypes binding of libzfact (include/zfact.h): argument marshalling only.

Every step of the factorization runs in the library's CUDA kernels; this
module converts torch tensors / numpy arrays into pointers and sizes and
turns status codes into exceptions.  It never falls back to a CPU
implementation: if the library is missing it raises.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libzfact.so")

OK = 0
ERR_ARG, ERR_CUDA, ERR_NOMEM, ERR_NONFINITE, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_UNSUPPORTED = 1, 2, 3, 4, 5, 6, 7
WARN_NONCONTRACTIVE = 100

PRECISION = {"fp64": 0, "fp32": 1, "bf16": 3, "fp16": 4, "fp16_split": 5, "bf16_split": 6, "fp16_half": 7}
REFINE_MODE = {"native": 0, "ozaki": 1, "fp32": 2}
EMULATION = {"auto": 0, "slices": 1, "wide": 2}
MLP_NPARAMS = 5573

EXPORTED = (
    "zfact_default_opts", "zfact_create", "zfact_destroy", "zfact_last_error", "zfact_refine",
    "zfact_refine_batched", "zfact_features", "zfact_mlp_forward", "zfact_mlp_backward",
    "zfact_mlp_adam", "zfact_propose", "zfact_gemm", "zfact_split", "zfact_residual",
    "zfact_set_profiling", "zfact_kernel_stats", "zfact_residual_noalloc", "zfact_congruence",
    "zfact_set_workspace_limit", "zfact_selftest_timeout", "zfact_set_emulation", "zfact_set_loop_graphs",
)


class ZfactError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("zfact error %d: %s" % (code, msg))
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("nmax", ctypes.c_int), ("refine_steps", ctypes.c_int), ("refine_mode", ctypes.c_int),
                ("stop_rule", ctypes.c_int), ("tol", ctypes.c_double), ("fixed_iters", ctypes.c_int),
                ("final_residual", ctypes.c_int), ("tile_cfg", ctypes.c_int), ("start_scale", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("refine_iters", ctypes.c_int), ("hist_len", ctypes.c_int),
                ("warn", ctypes.c_int), ("launches", ctypes.c_int), ("resid_f", ctypes.c_double),
                ("ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


_lib = None


def load(path: Optional[str] = None):
    """Load libzfact.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError("libzfact.so not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    P, I, I64, D, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_float
    lib.zfact_default_opts.argtypes = [ctypes.POINTER(Opts)]
    lib.zfact_default_opts.restype = None
    lib.zfact_create.argtypes = [ctypes.POINTER(P), I, P]
    lib.zfact_destroy.argtypes = [P]
    lib.zfact_destroy.restype = None
    lib.zfact_last_error.argtypes = [P]
    lib.zfact_last_error.restype = ctypes.c_char_p
    lib.zfact_refine.argtypes = [P, P, P, I64, I, I, ctypes.POINTER(Opts), P, P, I, ctypes.POINTER(Info)]
    lib.zfact_refine_batched.argtypes = [P, I, P, P, P, P, I, ctypes.POINTER(Opts), P, P, I, P, P]
    lib.zfact_features.argtypes = [P, P, I64, P]
    lib.zfact_mlp_forward.argtypes = [P, P, P, P, P, I, P]
    lib.zfact_mlp_backward.argtypes = [P, P, P, P, P, P, P, I, F, P, ctypes.POINTER(D)]
    lib.zfact_mlp_adam.argtypes = [P, P, P, P, P, I, I, F, F, F, F]
    lib.zfact_propose.argtypes = [P, P, I64, P, P, P, ctypes.POINTER(D), ctypes.POINTER(I)]
    lib.zfact_gemm.argtypes = [P, I, I64, P, D, P, D, P]
    lib.zfact_split.argtypes = [P, I, P, I64, D, P, P]
    lib.zfact_residual.argtypes = [P, I, P, P, I64, P, ctypes.POINTER(D)]
    lib.zfact_set_profiling.argtypes = [P, I]
    lib.zfact_kernel_stats.argtypes = [P, P, I, ctypes.POINTER(I), I]
    lib.zfact_residual_noalloc.argtypes = [P, P, I64, P, P, P]
    lib.zfact_congruence.argtypes = [P, P, P, I64, I, I, P]
    lib.zfact_set_workspace_limit.argtypes = [P, I64]
    lib.zfact_selftest_timeout.argtypes = [P]
    lib.zfact_set_emulation.argtypes = [P, I]
    lib.zfact_set_loop_graphs.argtypes = [P, I]
    for name in EXPORTED:
        if getattr(lib, name).restype is ctypes.c_int or name in ("zfact_default_opts", "zfact_destroy",
                                                                      "zfact_last_error"):
            continue
        getattr(lib, name).restype = I
    _lib = lib
    return lib


def _ptr(a):
    """Raw pointer of a torch tensor (device or host) or numpy array (host)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(type(a))


def _check_f64(a, n, name):
    if a is None:
        return
    dt = getattr(a, "dtype", None)
    ok = (str(dt) in ("torch.float64", "float64"))
    if not ok:
        raise TypeError("%s must be float64, got %s" % (name, dt))
    if tuple(a.shape) != (n, n):
        raise ValueError("%s must be %dx%d, got %s" % (name, n, n, tuple(a.shape)))


def make_opts(**kw) -> Opts:
    o = Opts()
    load().zfact_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if v is None:
            continue
        if k == "refine_mode" and isinstance(v, str):
            v = REFINE_MODE[v]
        setattr(o, k, v)
    return o


@dataclass
class Result:
    Z: object
    hist: np.ndarray
    info: dict
    status: int


class Context:
    """One zfact_ctx on a CUDA device (optionally bound to a torch stream)."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load()
        h = ctypes.c_void_p()
        sp = None
        if stream is not None:
            sp = getattr(stream, "cuda_stream", stream)
        rc = self.lib.zfact_create(ctypes.byref(h), int(device), sp)
        if rc != OK:
            raise ZfactError(rc, "zfact_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.zfact_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def last_error(self) -> str:
        return self.lib.zfact_last_error(self.h).decode()

    def _raise(self, rc, allow=(OK, WARN_NONCONTRACTIVE)):
        if rc not in allow:
            raise ZfactError(rc, self.last_error())

    @staticmethod
    def _ready(*objs):
        """Wait for the current torch stream of every CUDA tensor passed to a call.

        The library queues its work on the context's stream, which is not ordered after the
        stream torch wrote the inputs on (nor after torch work still reading a recycled output
        block).  Every call is synchronous, so a host wait costs nothing the call would not."""
        seen = set()
        stack = list(objs)
        while stack:
            a = stack.pop()
            if isinstance(a, (list, tuple)):
                stack.extend(a)
            elif getattr(a, "is_cuda", False) and a.device not in seen:
                import torch
                seen.add(a.device)
                torch.cuda.current_stream(a.device).synchronize()

    # ------------------------------------------------------------ refine
    def refine(self, S, Z0=None, order: int = 2, precision: str = "fp64", Z=None, hist_cap: int = 128,
               raise_on_error: bool = True, **opts) -> Result:
        """zfact_refine: S (N x N float64, torch device/host tensor or numpy array)."""
        n = int(S.shape[0])
        _check_f64(S, n, "S")
        _check_f64(Z0, n, "Z0")
        if Z is None:
            if hasattr(S, "new_empty"):
                Z = S.new_empty((n, n))
            else:
                Z = np.empty((n, n))
        _check_f64(Z, n, "Z")
        o = make_opts(**opts)
        hist = np.full(hist_cap, np.nan)
        info = Info()
        self._ready(S, Z0, Z)
        rc = self.lib.zfact_refine(self.h, _ptr(S), _ptr(Z0), n, int(order), PRECISION[precision],
                                   ctypes.byref(o), _ptr(Z), hist.ctypes.data, int(hist_cap),
                                   ctypes.byref(info))
        if raise_on_error:
            self._raise(rc)
        return Result(Z, hist[:info.hist_len].copy(), info.as_dict(), rc)

    # ------------------------------------------------------------ batched
    def refine_batched(self, S_list: Sequence, Z0_list=None, orders=None, precision: str = "bf16",
                       Z_list=None, hist_cap: int = 64, raise_on_error: bool = True, **opts):
        import torch
        count = len(S_list)
        ns = np.array([int(s.shape[0]) for s in S_list], dtype=np.int64)
        if Z_list is None:
            Z_list = [torch.empty_like(s) for s in S_list]
        if orders is None:
            orders = [2] * count
        sp = (ctypes.c_void_p * count)(*[_ptr(s) for s in S_list])
        zp = (ctypes.c_void_p * count)(*[_ptr(z) for z in Z_list])
        z0p = None
        if Z0_list is not None:
            z0p = (ctypes.c_void_p * count)(*[_ptr(z) if z is not None else None for z in Z0_list])
        ords = np.ascontiguousarray(orders, dtype=np.int32)
        hist = np.full((count, hist_cap), np.nan)
        infos = (Info * count)()
        status = np.zeros(count, dtype=np.int32)
        o = make_opts(**opts)
        self._ready(S_list, Z_list, Z0_list)
        rc = self.lib.zfact_refine_batched(self.h, count, sp, z0p, ns.ctypes.data, ords.ctypes.data,
                                           PRECISION[precision], ctypes.byref(o), zp, hist.ctypes.data,
                                           hist_cap, infos, status.ctypes.data)
        if raise_on_error or rc not in (OK, WARN_NONCONTRACTIVE, ERR_NONFINITE, ERR_NOT_CONVERGED):
            self._raise(rc)
        return Z_list, hist, [i.as_dict() for i in infos], status

    # ------------------------------------------------------------ workspace cap, self-test
    def set_workspace_limit(self, nbytes: int = 0):
        """zfact_set_workspace_limit: cap the device workspace (0 = no cap)."""
        self._raise(self.lib.zfact_set_workspace_limit(self.h, int(nbytes)))

    def set_loop_graphs(self, on: bool = True):
        """zfact_set_loop_graphs: run the bulk's updates after the first as one device-driven CUDA graph
        (default) or one by one from the host."""
        self._raise(self.lib.zfact_set_loop_graphs(self.h, int(bool(on))))

    def set_emulation(self, scheme: str = "auto"):
        """zfact_set_emulation: "auto" (CRT residues, sixteen moduli or up to 24 where the rows need more
        bits, else slices), "slices", or "wide" (the same as "auto")."""
        self._raise(self.lib.zfact_set_emulation(self.h, EMULATION[scheme] if isinstance(scheme, str) else int(scheme)))

    def selftest_timeout(self) -> int:
        """zfact_selftest_timeout: returns the status (ZFACT_ERR_TIMEOUT = 6 when the path works)."""
        return int(self.lib.zfact_selftest_timeout(self.h))

    # ------------------------------------------------------------ per-kernel timing
    def set_profiling(self, on: bool = True):
        self._raise(self.lib.zfact_set_profiling(self.h, int(bool(on))))

    def kernel_stats(self, reset: bool = True):
        cap = 64
        arr = (KStat * cap)()
        n = ctypes.c_int()
        self._raise(self.lib.zfact_kernel_stats(self.h, arr, cap, ctypes.byref(n), int(bool(reset))))
        return [{"name": arr[i].name.decode(), "launches": arr[i].launches, "ms": arr[i].ms,
                 "flops": arr[i].flops, "bytes": arr[i].bytes} for i in range(min(n.value, cap))]

    # ------------------------------------------------------------ steps
    def gemm(self, A, B, precision: str = "bf16", scale_a: float = 1.0, scale_b: float = 1.0, C=None):
        n = int(A.shape[0])
        C = A.new_empty((n, n)) if C is None else C
        self._ready(A, B, C)
        rc = self.lib.zfact_gemm(self.h, PRECISION[precision], n, _ptr(A), scale_a, _ptr(B), scale_b, _ptr(C))
        self._raise(rc)
        return C

    def split(self, A, precision: str = "fp16", scale: float = 1.0):
        import torch
        n = int(A.numel())
        hi = torch.empty(n, dtype=torch.int16, device=A.device)
        lo = torch.empty(n, dtype=torch.int16, device=A.device)
        self._ready(A, hi, lo)
        rc = self.lib.zfact_split(self.h, PRECISION[precision], _ptr(A), n, scale, _ptr(hi), _ptr(lo))
        self._raise(rc)
        return hi, lo

    def residual(self, S, Z, mode: str = "native", D=None):
        n = int(S.shape[0])
        err = ctypes.c_double()
        self._ready(S, Z, D)
        rc = self.lib.zfact_residual(self.h, REFINE_MODE[mode], _ptr(S), _ptr(Z), n, _ptr(D), ctypes.byref(err))
        self._raise(rc)
        return err.value

    def congruence(self, H, Z, precision: str = "fp64", mode: str = "ozaki", Hp=None):
        """zfact_congruence: H_perp = Z^T H Z (H symmetric), device or host operands."""
        n = int(H.shape[0])
        _check_f64(H, n, "H")
        _check_f64(Z, n, "Z")
        if Hp is None:
            Hp = H.new_empty((n, n)) if hasattr(H, "new_empty") else np.empty((n, n))
        _check_f64(Hp, n, "Hp")
        self._ready(H, Z, Hp)
        rc = self.lib.zfact_congruence(self.h, _ptr(H), _ptr(Z), n, PRECISION[precision], REFINE_MODE[mode],
                                       _ptr(Hp))
        self._raise(rc)
        return Hp

    # ------------------------------------------------------------ learned start
    def features(self, S):
        feat = np.zeros(16, dtype=np.float32)
        self._ready(S)
        rc = self.lib.zfact_features(self.h, _ptr(S), int(S.shape[0]), feat.ctypes.data)
        self._raise(rc)
        return feat

    def mlp_forward(self, params, mean, std, x, y=None):
        import torch
        b = int(x.shape[0])
        y = torch.empty((b, 5), dtype=torch.float32, device=x.device) if y is None else y
        self._ready(params, mean, std, x, y)
        rc = self.lib.zfact_mlp_forward(self.h, _ptr(params), _ptr(mean), _ptr(std), _ptr(x), b, _ptr(y))
        self._raise(rc)
        return y

    def mlp_backward(self, params, mean, std, x, t_scale, t_order, w_order=1.0, grad=None):
        import torch
        b = int(x.shape[0])
        grad = torch.empty(MLP_NPARAMS, dtype=torch.float32, device=x.device) if grad is None else grad
        loss = ctypes.c_double()
        self._ready(params, mean, std, x, t_scale, t_order, grad)
        rc = self.lib.zfact_mlp_backward(self.h, _ptr(params), _ptr(mean), _ptr(std), _ptr(x), _ptr(t_scale),
                                         _ptr(t_order), b, float(w_order), _ptr(grad), ctypes.byref(loss))
        self._raise(rc)
        return grad, loss.value

    def mlp_adam(self, params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self._ready(params, grad, m, v)
        rc = self.lib.zfact_mlp_adam(self.h, _ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(params.numel()),
                                     int(step), float(lr), float(beta1), float(beta2), float(eps))
        self._raise(rc)

    def propose(self, S, params, mean, std):
        s = ctypes.c_double()
        m = ctypes.c_int()
        self._ready(S, params, mean, std)
        rc = self.lib.zfact_propose(self.h, _ptr(S), int(S.shape[0]), _ptr(params), _ptr(mean), _ptr(std),
                                    ctypes.byref(s), ctypes.byref(m))
        self._raise(rc)
        return s.value, m.value
