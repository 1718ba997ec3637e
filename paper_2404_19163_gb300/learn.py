"""Learned start proposal: labels from the method itself, training on the library's
MLP kernels, and evaluation against the plain schedule.

For every training matrix the method is run (grouped launches, BF16 hi/lo split bulk,
Algorithm 2 stop) from Z0 = f s0 I for each start factor f of a grid and each order m;
the label is the (f, m) of least modelled time of the whole factorization to
||I - Z^T S Z||_F / sqrt(N) <= tol:
  - bulk: one iteration costs (m + 4) N^3 multiply-adds on symmetric tiles (K1 2N^3,
    K2 N^3, the polynomial chain (m - 1) N^3, K4 2N^3), m + 2 kernel launches and one
    stop-test read-back:  ALPHA + BETA (m + 2) + (m + 4) N^3 / RATE  per iteration, run to
    the Algorithm 2 stop;
  - refinement: from the bulk's last Err e, the FP64-accurate updates needed to reach tol
    under e <- e^(m+1), each preceded by an FP64-accurate residual, plus the final residual
    (sliced products: 135 N^3 and 72 N^3 multiply-adds at the sliced-product rate, plus
    their launch overhead).
The network (16 -> 64 -> 64 -> 5, GELU) maps the features of S to log f and to logits of
m; zfact_propose applies it with the plain schedule (f = 1, m = 2) as fallback.

  python -m paper_2404_19163_gb300.learn --train 2000 --heldout 256 --out weights.npz
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import synth
from .zfact import MLP_NPARAMS, Context

F_GRID = (0.9, 1.0, 1.1, 1.25, 1.4, 1.6, 1.8, 2.0)
ORDERS = (2, 3, 4, 5)
ALPHA = 30e-6      # s per iteration: stop-test read-back
BETA = 8e-6        # s per kernel launch
RATE = 0.65e15     # multiply-adds per s of the split-BF16 bulk products (3 products each)
RATE_OZ = 0.85e15  # multiply-adds per s of the sliced FP64-accurate products
T_RES0 = 250e-6    # launch / read-back overhead of one FP64-accurate residual
T_UPD0 = 120e-6    # ... of one FP64-accurate update
TOL = 1e-12
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "propose_mlp.npz")


def instances(count: int, split: str, n_lo: int, n_hi: int):
    import torch
    return [torch.from_numpy(synth.proposal_instance(k, n_lo, n_hi, split)).cuda() for k in range(count)]


def features(ctx: Context, S_list):
    return np.stack([ctx.features(S) for S in S_list]).astype(np.float32)


def iter_time(n, m):
    """Modelled seconds of one bulk iteration of order m at size n."""
    return ALPHA + BETA * (m + 2) + (m + 4.0) * float(n) ** 3 / RATE


def work(hist, n, m, tau, tol=TOL):
    """Modelled seconds of the whole factorization (bulk to the Algorithm 2 stop, then the
    refinement to tol), inf if the bulk diverged or never got below tau."""
    h = np.asarray(hist, dtype=np.float64)
    if h.size == 0 or not np.all(np.isfinite(h)) or np.min(h) / math.sqrt(n) > tau:
        return math.inf
    k = h.size - 1
    n3 = float(n) ** 3
    t = 3.0 * n3 / RATE + k * iter_time(n, m)
    e, target, updates = float(h[-1]), tol * math.sqrt(n), 0
    while e > target and updates < 4:
        e = e ** (m + 1)
        updates += 1
    t += (updates + 1) * (T_RES0 + 135.0 * n3 / RATE_OZ) + updates * (T_UPD0 + 72.0 * n3 / RATE_OZ)
    return t


def label(ctx: Context, S_list, feats, tau=1e-4, precision="bf16_split", nmax=30):
    """Run the method over the (f, m) grid; returns (log f*, index of m*, work table)."""
    import torch
    B = len(S_list)
    ns = [int(S.shape[0]) for S in S_list]
    s0 = np.exp(-0.5 * feats[:, 1].astype(np.float64))
    table = np.full((B, len(F_GRID), len(ORDERS)), math.inf)
    for fi, f in enumerate(F_GRID):
        Z0 = [torch.eye(n, dtype=torch.float64, device="cuda") * (f * s0[i]) for i, n in enumerate(ns)]
        for mi, m in enumerate(ORDERS):
            _, hist, infos, status = ctx.refine_batched(S_list, Z0, orders=[m] * B, precision=precision,
                                                        hist_cap=nmax + 2, nmax=nmax, final_residual=0,
                                                        raise_on_error=False)
            for i in range(B):
                table[i, fi, mi] = work(hist[i][:infos[i]["hist_len"]], ns[i], m, tau)
        del Z0
    flat = table.reshape(B, -1)
    best = np.argmin(flat, axis=1)
    ok = np.isfinite(flat[np.arange(B), best])
    fi, mi = np.unravel_index(best, (len(F_GRID), len(ORDERS)))
    y_scale = np.log(np.asarray(F_GRID))[fi].astype(np.float32)
    y_order = mi.astype(np.int32)
    # instances no grid point solved keep the plain schedule as their label
    y_scale[~ok] = 0.0
    y_order[~ok] = 0
    return y_scale, y_order, table


def init_params(seed=0):
    g = np.random.default_rng(seed)
    sizes = (16, 64, 64, 5)
    out = []
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        out.append(g.standard_normal(fo * fi) * math.sqrt(2.0 / (fi + fo)))
        out.append(np.zeros(fo))
    p = np.concatenate(out).astype(np.float32)
    assert p.size == MLP_NPARAMS
    return p


def train(ctx: Context, X, y_scale, y_order, steps=3000, lr=3e-3, w_order=1.0, seed=0, log_every=0):
    """Full-batch Adam on the library's forward/backward/Adam kernels.  Returns
    (params, mean, std, loss history) with params/mean/std as device tensors."""
    import torch
    X = np.asarray(X, dtype=np.float32)
    mean = X.mean(axis=0)
    std = X.std(axis=0) + 1e-6
    dev = lambda a, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)
    P = dev(init_params(seed))
    M = torch.zeros_like(P)
    V = torch.zeros_like(P)
    Xd, mu, sd = dev(X), dev(mean), dev(std)
    ts, to = dev(y_scale), dev(y_order, torch.int32)
    losses = []
    for step in range(1, steps + 1):
        grad, loss = ctx.mlp_backward(P, mu, sd, Xd, ts, to, w_order)
        ctx.mlp_adam(P, grad, M, V, step, lr=lr)
        losses.append(loss)
        if log_every and step % log_every == 0:
            print("step %d loss %.5f" % (step, loss), flush=True)
    return P, mu, sd, losses


def evaluate(ctx: Context, S_list, P, mu, sd, precision="bf16_split"):
    """Plain schedule vs proposal on each matrix: device ms of the bulk alone (to the
    Algorithm 2 stop) and of the full path to tol = max(1e-12, 1e-16 cond(S)) (bulk +
    refinement + FP64-accurate final residual), and the bulk iterations."""
    import torch
    rows = []
    for S in S_list:
        n = int(S.shape[0])
        lam = torch.linalg.eigvalsh(S)
        tol = max(1e-12, 1e-16 * float(lam[-1] / lam[0]))
        s, m = ctx.propose(S, P, mu, sd)
        Z0 = torch.eye(n, dtype=torch.float64, device="cuda") * s
        row = {"n": n, "tol": tol, "m": m}
        for tag, z0, mm in (("plain", None, 2), ("prop", Z0, m)):
            rb = ctx.refine(S, z0, order=mm, precision=precision, refine_steps=0, final_residual=0,
                            raise_on_error=False)
            rf = ctx.refine(S, z0, order=mm, precision=precision, tol=tol, raise_on_error=False)
            ms, ok = rf.info["ms"], rf.status in (0, 100)
            if tag == "prop" and not ok:
                # the FP64-accurate final residual rejected the proposed start: fall back to the
                # plain schedule and charge both runs
                rp = ctx.refine(S, None, order=2, precision=precision, tol=tol, raise_on_error=False)
                ms, ok = ms + rp.info["ms"], rp.status in (0, 100)
                row["fallback"] = True
            row.update({tag + "_bulk_ms": rb.info["ms"], tag + "_iters": rb.info["iters"],
                        tag + "_ms": ms, tag + "_ok": ok})
        rows.append(row)
    return rows


def save(path, P, mu, sd, meta):
    np.savez(path, params=P.cpu().numpy(), mean=mu.cpu().numpy(), std=sd.cpu().numpy(),
             meta=json.dumps(meta))


def load(path=WEIGHTS):
    import torch
    z = np.load(path)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float32)
    return dev(z["params"]), dev(z["mean"]), dev(z["std"]), json.loads(str(z["meta"]))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--heldout", type=int, default=256)
    ap.add_argument("--n-lo", type=int, default=128)
    ap.add_argument("--n-hi", type=int, default=1536)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--tau", type=float, default=1e-4)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--chunk", type=int, default=500)
    args = ap.parse_args()
    t0 = time.time()
    with Context(0) as ctx:
        feats, ys, yo = [], [], []
        for c0 in range(0, args.train, args.chunk):
            Ss = [__import__("torch").from_numpy(synth.proposal_instance(k, args.n_lo, args.n_hi, "train")).cuda()
                  for k in range(c0, min(args.train, c0 + args.chunk))]
            f = features(ctx, Ss)
            a, b, _ = label(ctx, Ss, f, tau=args.tau)
            feats.append(f)
            ys.append(a)
            yo.append(b)
            del Ss
        X = np.concatenate(feats)
        y_scale = np.concatenate(ys)
        y_order = np.concatenate(yo)
        t_label = time.time() - t0
        P, mu, sd, losses = train(ctx, X, y_scale, y_order, steps=args.steps)
        Sh = instances(args.heldout, "heldout", args.n_lo, args.n_hi)
        rows = evaluate(ctx, Sh, P, mu, sd)
        plain = sum(r["plain_ms"] for r in rows)
        prop = sum(r["prop_ms"] for r in rows)
        plain_b = sum(r["plain_bulk_ms"] for r in rows)
        prop_b = sum(r["prop_bulk_ms"] for r in rows)
        meta = {"train": args.train, "heldout": args.heldout, "n_range": [args.n_lo, args.n_hi], "tau": args.tau,
                "label_seconds": round(t_label, 1), "final_loss": losses[-1],
                "label_order_hist": np.bincount(y_order, minlength=4).tolist(),
                "label_f_mean": float(np.exp(y_scale).mean()),
                "heldout_plain_ms": plain, "heldout_proposed_ms": prop,
                "heldout_plain_bulk_ms": plain_b, "heldout_proposed_bulk_ms": prop_b,
                "heldout_order_hist": np.bincount([r["m"] - 2 for r in rows], minlength=4).tolist(),
                "heldout_plain_iters": float(np.mean([r["plain_iters"] for r in rows])),
                "heldout_proposed_iters": float(np.mean([r["prop_iters"] for r in rows])),
                "heldout_converged": [sum(r["plain_ok"] for r in rows), sum(r["prop_ok"] for r in rows)],
                "heldout_fallbacks": sum(1 for r in rows if r.get("fallback"))}
        save(args.out, P, mu, sd, meta)
        print(json.dumps(meta), flush=True)


if __name__ == "__main__":
    main()
