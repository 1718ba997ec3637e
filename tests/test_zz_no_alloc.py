"""zfact_residual_noalloc against the allocating zfact_residual and the FP64 oracle.

Some callers cannot allocate device memory where they need the residual: an
application whose own pool owns the whole device, or a latency-critical step
loop that cannot take the device synchronisation a cudaMalloc may cause.  For
them zfact_residual_noalloc keeps its scratch in one static device array.  It
must return the same d = I - Z^T S Z and ||d||_F as zfact_residual, on every
call, even though consecutive calls reuse (and leave behind) that scratch.
This file is collected last so that a failure here never hides another test."""
import ctypes

import numpy as np
import pytest

import oracle

from paper_2404_19163_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL = 1e-12


def test_noalloc_residual_matches_zfact_residual_two_calls():
    import torch
    from paper_2404_19163_gb300 import Context, build, load
    build.build()
    lib = load()
    g = np.random.default_rng(31)
    with Context(0) as ctx:
        # two calls in a row with different sizes and inputs: stale scratch would show
        for n in (1024, 333):
            S, Q, lam = synth.householder_spd(n, seed=n)
            Z = (Q * lam ** -0.5) @ Q.T + 0.01 * g.standard_normal((n, n))
            St = torch.from_numpy(S).cuda()
            Zt = torch.from_numpy(Z).cuda()
            D_ref = torch.empty_like(St)
            err_ref = ctx.residual(St, Zt, "native", D=D_ref)
            D = torch.full_like(St, float("nan"))
            err = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            rc = lib.zfact_residual_noalloc(St.data_ptr(), Zt.data_ptr(), n, D.data_ptr(), err.data_ptr(), None)
            assert rc == 0
            torch.cuda.synchronize()
            d_ref = D_ref.cpu().numpy()
            assert np.linalg.norm(D.cpu().numpy() - d_ref) <= RTOL * max(1.0, np.linalg.norm(d_ref))
            assert abs(err.item() - err_ref) <= RTOL * max(1.0, err_ref)
            # and against the oracle's FP64 d = I - Z^T S Z, element by element: two FP64
            # evaluations of the same products differ by rounding on the scale of |Z|^T |S| |Z|
            d_or, err_or = oracle.residual(S, Z)
            scale = float(np.max(np.abs(Z).T @ (np.abs(S) @ np.abs(Z))))
            assert float(np.max(np.abs(D.cpu().numpy() - d_or))) <= 1e-13 * scale
            assert abs(err.item() - err_or) <= 1e-13 * scale * n


def test_noalloc_rejects_oversize():
    import torch
    from paper_2404_19163_gb300 import build, load
    build.build()
    lib = load()
    x = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert lib.zfact_residual_noalloc(x.data_ptr(), x.data_ptr(), 1025, x.data_ptr(), e.data_ptr(), None) == 1
    assert lib.zfact_residual_noalloc(x.data_ptr(), x.data_ptr(), 0, x.data_ptr(), e.data_ptr(), None) == 1
