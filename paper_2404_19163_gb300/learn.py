"""Learned start proposal: labels from the method itself, training on the library's
MLP kernels, and evaluation against the plain schedule.

For every training matrix the method is run (grouped launches, BF16 hi/lo split bulk,
Algorithm 2 stop) from Z0 = f s0 I for each start factor f of a grid and each order m;
the label is the (f, m) of least modelled time of the whole factorization to
||I - Z^T S Z||_F / sqrt(N) <= tol:
  - bulk: one iteration of order m runs (m + 4) N^3 multiply-adds on symmetric tiles (K1 2N^3,
    K2 N^3, the polynomial chain (m - 1) N^3, K4 2N^3) in m + 2 tensor-core launches plus a
    stop-test read-back:  ALPHA + BETA (m + 2) + (m + 4) N^3 C_BULK  per iteration, run to the
    Algorithm 2 stop;
  - refinement: from the bulk's last Err e, the FP64-accurate updates needed to reach tol
    under e <- e^(m'+1) / N^(m'/2) (m' the refinement's order: the lowest whose estimated error term
    is at most half the target, else m), each preceded by an FP64-accurate residual, plus the final residual:
    T_RES0 + C_RES N^3 per residual and T_UPD0 + C_UPD N^3 per update (CRT residue products).
The constants are GB300 measurements of the library's own kernels (bulk products and CRT
refinement of the N = 4096 factorization; per-launch and read-back latencies of small N).
The network (16 -> 64 -> 64 -> 5, GELU) maps the features of S to log f and to logits of
m; zfact_propose applies it with the plain schedule (f = 1, m = 2) as fallback.

  python -m paper_2404_19163_gb300.learn --train 20000 --heldout 512 --save-dir DIR
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

# start factors f >= 1: the Gershgorin scale puts every eigenvalue of X0 = s0^2 S in (0, 1], so a
# smaller f only lowers the smallest one
F_GRID = (1.0, 1.1, 1.25, 1.4, 1.6, 1.8, 2.0)
ORDERS = (2, 3, 4, 5)
ALPHA = 30e-6      # s per bulk iteration: the stop-test read-back
BETA = 8e-6        # s per kernel launch
C_BULK = 2.4e-15   # s per N^3 multiply-add unit of the split-BF16 bulk (3 BF16 products each)
T_RES0 = 200e-6    # launches and read-back of one FP64-accurate residual
C_RES = 5.0e-14    # s per N^3 of one FP64-accurate residual (two CRT products, residues, reconstruction)
T_UPD0 = 100e-6    # launches of one FP64-accurate update
C_UPD = 2.2e-14    # s per N^3 of one FP64-accurate update Z + Z Q
TOL = 1e-12
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "propose_mlp.npz")
PACK_BYTES = 52    # bytes per (packed row x leading dimension) element of the grouped mode's buffers


def instances(count: int, split: str, n_lo: int, n_hi: int, start: int = 0):
    """Matrices k = start .. start + count - 1 of the proposal family, built on the GPU."""
    return [synth.proposal_instance_torch(k, n_lo, n_hi, split) for k in range(start, start + count)]


def features(ctx: Context, S_list):
    return np.stack([ctx.features(S) for S in S_list]).astype(np.float32)


def default_model():
    """Cost model from the constants above: per order m, one bulk iteration costs
    iter[m] = (a, b) -> a + b N^3 seconds; an FP64-accurate residual res = (a, b) and update upd = (a, b)."""
    return {"iter": {m: (ALPHA + BETA * (m + 2), (m + 4.0) * C_BULK) for m in ORDERS},
            "res": (T_RES0, C_RES), "upd": (T_UPD0, C_UPD), "source": "constants"}


def iter_time(n, m, model=None):
    """Modelled seconds of one bulk iteration of order m at size n."""
    a, b = (model or default_model())["iter"][m]
    return a + b * float(n) ** 3


def work(hist, n, m, tau, tol=TOL, model=None):
    """Modelled seconds of the whole factorization (bulk to the Algorithm 2 stop, then the
    refinement to tol), inf if the bulk diverged or never got below tau."""
    model = model or default_model()
    h = np.asarray(hist, dtype=np.float64)
    if h.size == 0 or not np.all(np.isfinite(h)) or np.min(h) / math.sqrt(n) > tau:
        return math.inf
    k = h.size - 1
    n3 = float(n) ** 3
    t = k * iter_time(n, m, model)
    e, target, updates = float(h[-1]), tol * math.sqrt(n), 0
    while e > target and updates < 4:
        # the refinement's order, as the library picks it: the lowest m' >= 2 whose estimated error term
        # e^(m'+1) / N^(m'/2) is at most half the target, else m
        mr = next((q for q in range(2, 6) if e ** (q + 1) / float(n) ** (0.5 * q) <= 0.5 * target), m)
        e = e ** (mr + 1) / float(n) ** (0.5 * mr)
        updates += 1
    (r0, r1), (u0, u1) = model["res"], model["upd"]
    t += (updates + 1) * (r0 + r1 * n3) + updates * (u0 + u1 * n3)
    return t


def _fit(ns, ts):
    """Least-squares a + b N^3 to the times ts at sizes ns, in relative terms (every size counts)."""
    ns = np.asarray(ns, dtype=np.float64)
    ts = np.asarray(ts, dtype=np.float64)
    A = np.stack([1.0 / ts, ns ** 3 / ts], axis=1)
    (a, b), *_ = np.linalg.lstsq(A, np.ones_like(ts), rcond=None)
    return float(max(a, 0.0)), float(max(b, 0.0))


def calibrate(ctx: Context, sizes=(128, 256, 512, 1024, 2048, 4096), reps=3, precision="bf16_split", log=print):
    """Measure the cost model on this GPU with the library's own runs: for each size and order, the
    device time of 2 and of 6 fixed bulk iterations (the difference is four iterations); for each size,
    an FP64-accurate residual alone, and a full factorization minus its bulk (one update and two
    residuals).  Matrices: jittered cubic Gaussian overlaps (the proposal family's middle)."""
    import torch

    def best(f):
        return min(f() for _ in range(reps))

    it = {m: [] for m in ORDERS}
    res, upd = [], []
    for n in sizes:
        side = int(math.ceil(n ** (1.0 / 3.0)))
        S = synth.gaussian_overlap_torch(synth.cubic_sites(side, 2.5, 0.1, 7, workload=5)[:n])
        for m in ORDERS:
            t = [best(lambda k=k: ctx.refine(S, None, order=m, precision=precision, fixed_iters=k, refine_steps=0,
                                              final_residual=0).info["ms"]) for k in (2, 6)]
            it[m].append(max(t[1] - t[0], 1e-3) / 4.0 * 1e-3)
        rb = ctx.refine(S, None, order=2, precision=precision, refine_steps=0, final_residual=0)
        Z = rb.Z.clone()

        def resid_ms():
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            ctx.residual(S, Z, "ozaki")
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)

        r = best(resid_ms) * 1e-3
        full = best(lambda: ctx.refine(S, None, order=2, precision=precision, tol=TOL).info["ms"])
        bulk = best(lambda: ctx.refine(S, None, order=2, precision=precision, refine_steps=0,
                                       final_residual=0).info["ms"])
        res.append(r)
        upd.append(max((full - bulk) * 1e-3 - 2.0 * r, 0.1 * r))
        log("calibrate N=%d: iteration ms %s, residual %.3f ms, update %.3f ms" %
            (n, " ".join("m%d %.3f" % (m, it[m][-1] * 1e3) for m in ORDERS), r * 1e3, upd[-1] * 1e3))
    return {"iter": {m: _fit(sizes, it[m]) for m in ORDERS}, "res": _fit(sizes, res), "upd": _fit(sizes, upd),
            "source": "measured", "sizes": list(sizes)}


def label(ctx: Context, S_list, feats, tau=1e-4, precision="bf16_split", nmax=30, model=None):
    """Run the method over the (f, m) grid; returns (log f*, index of m*, work table)."""
    import torch
    B = len(S_list)
    ns = [int(S.shape[0]) for S in S_list]
    s0 = np.exp(-0.5 * feats[:, 1].astype(np.float64))
    table = np.full((B, len(F_GRID), len(ORDERS)), math.inf)
    Z_out = [torch.empty_like(S) for S in S_list]
    for fi, f in enumerate(F_GRID):
        Z0 = [torch.eye(n, dtype=torch.float64, device="cuda") * (f * s0[i]) for i, n in enumerate(ns)]
        for mi, m in enumerate(ORDERS):
            _, hist, infos, status = ctx.refine_batched(S_list, Z0, orders=[m] * B, precision=precision,
                                                        Z_list=Z_out, hist_cap=nmax + 2, nmax=nmax,
                                                        final_residual=0, raise_on_error=False)
            for i in range(B):
                table[i, fi, mi] = work(hist[i][:infos[i]["hist_len"]], ns[i], m, tau, model=model)
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


def size_batches(ns, budget_bytes=24 << 30, max_count=512):
    """Groups of instance indices, smallest N first, for grouped label runs: the grouped mode packs
    every instance of a call with the largest N's leading dimension, so instances of similar N go
    together, each group within a memory budget."""
    rup = lambda x, m: (x + m - 1) // m * m
    batches, cur, rows = [], [], 0
    for i in np.argsort(np.asarray(ns), kind="stable"):
        n = int(ns[i])
        r = rows + rup(n, 256)
        if cur and (r * rup(n, 64) * PACK_BYTES > budget_bytes or len(cur) >= max_count):
            batches.append(cur)
            cur, r = [], rup(n, 256)
        cur.append(int(i))
        rows = r
    if cur:
        batches.append(cur)
    return batches


def label_set(ctx: Context, count: int, n_lo: int, n_hi: int, tau=1e-4, save_dir=None, log=print, model=None,
              max_seconds=0.0):
    """Features and labels of training matrices 0 .. count-1, grouped by size.  With save_dir,
    every finished group is kept in save_dir/labels_<first>.npz and skipped on a rerun.  With
    max_seconds > 0 no new group starts after that many seconds; returns (X, y_scale, y_order, done)."""
    import torch
    t0 = time.time()
    sites = [synth.proposal_sites(k, n_lo, n_hi, "train") for k in range(count)]
    ns = np.array([p.shape[0] for p, _ in sites])
    log("sites for %d matrices in %.1f s; N in [%d, %d], sum N^3 = %.3g" %
        (count, time.time() - t0, ns.min(), ns.max(), float(np.sum(ns.astype(np.float64) ** 3))))
    X = np.zeros((count, 16), np.float32)
    ys = np.zeros(count, np.float32)
    yo = np.zeros(count, np.int32)
    batches = size_batches(ns)
    done = True
    for b, idx in enumerate(batches):
        path = os.path.join(save_dir, "labels_%06d.npz" % idx[0]) if save_dir else None
        if path and os.path.exists(path):
            z = np.load(path)
            if np.array_equal(z["idx"], idx):
                X[idx], ys[idx], yo[idx] = z["X"], z["ys"], z["yo"]
                continue
        if max_seconds > 0 and time.time() - t0 > max_seconds:
            done = False
            continue
        tb = time.time()
        Ss = [synth.gaussian_overlap_torch(*sites[k]) for k in idx]
        f = features(ctx, Ss)
        a, o, _ = label(ctx, Ss, f, tau=tau, model=model)
        X[idx], ys[idx], yo[idx] = f, a, o
        if path:
            np.savez(path, idx=np.asarray(idx), X=f, ys=a, yo=o)
        del Ss
        torch.cuda.empty_cache()
        log("group %d/%d: %d matrices, N %d..%d, %.1f s (total %.0f s)" %
            (b + 1, len(batches), len(idx), ns[idx[0]], ns[idx[-1]], time.time() - tb, time.time() - t0))
    return X, ys, yo, done


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


def tolerance(S):
    """max(1e-12, 1e-16 cond(S)): the FP64 floor of an ill-conditioned S sits above 1e-12."""
    import torch
    lam = torch.linalg.eigvalsh(S)
    return max(TOL, 1e-16 * float(lam[-1] / lam[0]))


def evaluate(ctx: Context, S_list, P, mu, sd, precision="bf16_split", tols=None, reps=2):
    """Plain schedule vs proposal on each matrix, measured: device ms of the bulk alone (to the
    Algorithm 2 stop) and of the full path to tol (bulk + refinement + FP64-accurate final residual),
    and the bulk iterations.  Both are cold starts Z0 = s I (no products for the first residual and
    update).  Each matrix first gets one untimed run of each schedule (workspace, tensor maps), then
    `reps` timed rounds in alternating order; the best time of each counts.  A proposal whose run the
    FP64-accurate final residual rejects falls back to the plain schedule and is charged both runs."""
    rows = []
    for k, S in enumerate(S_list):
        n = int(S.shape[0])
        tol = tolerance(S) if tols is None else tols[k]
        s, m = ctx.propose(S, P, mu, sd)
        sched = [("plain", 0.0, 2), ("prop", s, m)]
        for _, sc, mm in sched:
            ctx.refine(S, None, order=mm, precision=precision, tol=tol, start_scale=sc, raise_on_error=False)
        row = {"n": n, "tol": tol, "m": m, "s": s}
        for rep in range(reps):
            for tag, sc, mm in (sched if rep % 2 == 0 else sched[::-1]):
                rb = ctx.refine(S, None, order=mm, precision=precision, refine_steps=0, final_residual=0,
                                start_scale=sc, raise_on_error=False)
                rf = ctx.refine(S, None, order=mm, precision=precision, tol=tol, start_scale=sc, raise_on_error=False)
                row[tag + "_bulk_ms"] = min(row.get(tag + "_bulk_ms", math.inf), rb.info["ms"])
                row[tag + "_ms"] = min(row.get(tag + "_ms", math.inf), rf.info["ms"])
                row[tag + "_iters"] = rb.info["iters"]
                row[tag + "_refine"] = rf.info["refine_iters"]
                row[tag + "_ok"] = rf.status in (0, 100)
        if not row["prop_ok"]:
            row["prop_ms"] += row["plain_ms"]
            row["fallback"] = True
        rows.append(row)
    return rows


def summarize(rows):
    tot = lambda key: float(sum(r[key] for r in rows))
    out = {"count": len(rows),
           "plain_ms": tot("plain_ms"), "proposed_ms": tot("prop_ms"),
           "plain_bulk_ms": tot("plain_bulk_ms"), "proposed_bulk_ms": tot("prop_bulk_ms"),
           "plain_iters": float(np.mean([r["plain_iters"] for r in rows])),
           "proposed_iters": float(np.mean([r["prop_iters"] for r in rows])),
           "order_hist": np.bincount([r["m"] - 2 for r in rows], minlength=4).tolist(),
           "converged": [int(sum(r["plain_ok"] for r in rows)), int(sum(r["prop_ok"] for r in rows))],
           "fallbacks": int(sum(1 for r in rows if r.get("fallback"))),
           "fallbacks_where_plain_converged": int(sum(1 for r in rows if r.get("fallback") and r["plain_ok"]))}
    out["full_time_gain"] = 1.0 - out["proposed_ms"] / out["plain_ms"]
    out["bulk_time_gain"] = 1.0 - out["proposed_bulk_ms"] / out["plain_bulk_ms"]
    ok = [r for r in rows if r["plain_ok"]]
    if ok:
        out["full_time_gain_where_plain_converged"] = 1.0 - sum(r["prop_ms"] for r in ok) / sum(r["plain_ms"] for r in ok)
    # by size: where the bulk is a larger share of the path the proposal matters more
    bands = {}
    for lo, hi in ((0, 512), (512, 1536), (1536, 1 << 30)):
        sel = [r for r in rows if lo <= r["n"] < hi]
        if sel:
            p = sum(r["plain_ms"] for r in sel)
            bands["%d-%d" % (lo, min(hi, 4096))] = {"count": len(sel), "plain_ms": p,
                                                    "gain": 1.0 - sum(r["prop_ms"] for r in sel) / p}
    out["by_size"] = bands
    return out


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
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--heldout", type=int, default=512)
    ap.add_argument("--n-lo", type=int, default=128)
    ap.add_argument("--n-hi", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--tau", type=float, default=1e-4)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--save-dir", default=None, help="keep finished label groups here (resumable)")
    ap.add_argument("--label-only", action="store_true")
    ap.add_argument("--max-label-seconds", type=float, default=0.0,
                    help="start no new label group after this many seconds (rerun with the same --save-dir to go on)")
    ap.add_argument("--eval-only", default=None, metavar="WEIGHTS",
                    help="evaluate these trained weights on the held-out matrices (no labels, no training); "
                         "the weights file's metadata gets the new evaluation")
    args = ap.parse_args()
    if args.save_dir:
        os.makedirs(args.save_dir, exist_ok=True)
    log = lambda s: print(s, flush=True)
    t0 = time.time()
    if args.eval_only:
        with Context(0) as ctx:
            P, mu, sd, meta = load(args.eval_only)
            rows = []
            for k in range(args.heldout):
                rows += evaluate(ctx, instances(1, "heldout", args.n_lo, args.n_hi, start=k), P, mu, sd)
            meta["heldout_eval"] = summarize(rows)
            meta["heldout"] = args.heldout
            save(args.out, P, mu, sd, meta)
            if args.save_dir:
                with open(os.path.join(args.save_dir, "heldout_rows.json"), "w") as f:
                    json.dump(rows, f)
            log(json.dumps(meta))
        return
    with Context(0) as ctx:
        model = None
        mpath = os.path.join(args.save_dir, "cost_model.json") if args.save_dir else None
        if mpath and os.path.exists(mpath):
            with open(mpath) as f:
                model = json.load(f)
            model["iter"] = {int(k): tuple(v) for k, v in model["iter"].items()}
        if model is None:
            model = calibrate(ctx, log=log)
            if mpath:
                with open(mpath, "w") as f:
                    json.dump(model, f)
        log("cost model: %s" % json.dumps(model))
        X, y_scale, y_order, done = label_set(ctx, args.train, args.n_lo, args.n_hi, args.tau, args.save_dir, log,
                                              model, args.max_label_seconds)
        t_label = time.time() - t0
        if not done:
            log("labels incomplete: rerun with the same --save-dir")
            return
        if args.label_only:
            return
        P, mu, sd, losses = train(ctx, X, y_scale, y_order, steps=args.steps)
        log("trained: loss %.4f -> %.4f" % (losses[0], losses[-1]))
        rows = []
        for k in range(args.heldout):
            rows += evaluate(ctx, instances(1, "heldout", args.n_lo, args.n_hi, start=k), P, mu, sd)
        summ = summarize(rows)
        meta = {"train": args.train, "heldout": args.heldout, "n_range": [args.n_lo, args.n_hi], "tau": args.tau,
                "cost_model": model,
                "label_seconds": round(t_label, 1), "final_loss": losses[-1], "steps": args.steps,
                "label_order_hist": np.bincount(y_order, minlength=4).tolist(),
                "label_f_hist": np.bincount(np.argmin(np.abs(np.exp(y_scale)[:, None] - np.asarray(F_GRID)[None]),
                                                      axis=1), minlength=len(F_GRID)).tolist(),
                "heldout_eval": summ}
        save(args.out, P, mu, sd, meta)
        if args.save_dir:
            with open(os.path.join(args.save_dir, "heldout_rows.json"), "w") as f:
                json.dump(rows, f)
        log(json.dumps(meta))


if __name__ == "__main__":
    main()
