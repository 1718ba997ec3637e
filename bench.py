#!/usr/bin/env python
"""Benchmark of the inverse-overlap factorization Z Z^T = S^{-1} on GB300.

One step = one factorization of the workload to ||I - Z^T S Z||_F / sqrt(N) <= tol
(bulk iterations + Algorithm 3 refinement + the FP64-accurate final residual),
inputs resident on the device.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (default): N = 4096 Gaussian overlap, s-type sites exp(-r^2/2) on a
jittered 16^3 cubic lattice (spacing 2.5, jitter 0.1), cold start Z0 = I/sqrt(g_hi),
m = 2, BF16 tensor-core bulk with FP32 accumulation in the paper's split scheme
(h)(h)+(h)(l)+(l)(h) with BF16 hi/lo operands, then Algorithm 3's refinement with
d and Z + Z Q formed to FP64 accuracy on the tensor cores by modular (CRT) residue
products (error-free slicing where the moduli do not reach).
The single-instance path does not shard: with --gpus N every rank runs its own
replica (weak scaling) and value = max-over-ranks time / factorizations done.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms to ||I−ZᵀSZ||_F/√N≤tol per factorization; TFLOP/s & tensor-pipe % vs FP64 path"
UNIT = "ms"
TOL = 1e-12
# DRAM bytes per launch of the dominant kernel from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum, mean over the captured launches), valid only while the kernel's source is
# the one that was captured; otherwise the bench line reports traffic as null.
TRAFFIC = {
    "tc_gemm.crt": {"source": "paper_2404_19163_gb300/csrc/k_tc.cu", "sha1": "7de582aa31706a4e82353153ff56eded4536e13a",
                    "bytes_per_launch": 1.1328e9},
}
FP64_ITERS_WORKLOAD2 = 4   # updates the FP64 recursion needs on workload 2 (counted by the FP64 GPU path
                           # and by the oracle's own stop rule on the same input)


def captured_traffic(kernel):
    import hashlib
    t = TRAFFIC.get(kernel)
    if not t:
        return None
    try:
        with open(os.path.join(ROOT, t["source"]), "rb") as f:
            if hashlib.sha1(f.read()).hexdigest() != t["sha1"]:
                return None
    except OSError:
        return None
    return t["bytes_per_launch"]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def roofline_of(dom, total_ms, reasons, peaks, peak_src):
    """The `roofline` object of the dominant kernel family `dom` (name, launches, ms, flops, bytes from the
    library's per-launch events) over a timed region of total_ms with the sampler's throttle reasons.
    Tensor-core kernels: algorithmic TFLOP/s against the measured burst BF16 peak when the region lasts
    under a second without the power cap, else the sustained one; FP64 GEMMs: against the FP64 pipe;
    everything else: algorithmic GB/s against the measured copy bandwidth."""
    avg_ms = dom["ms"] / max(1, dom["launches"])
    fl = dom["flops"] / max(1, dom["launches"])
    by = dom["bytes"] / max(1, dom["launches"])
    capped = "sw_power_cap" in reasons
    if dom["name"].startswith("tc_gemm"):
        ach = fl / (avg_ms * 1e-3) / 1e12
        # burst peak for a kernel timed in a short region without power capping; the sustained
        # peak once the timed region lasts seconds or the sampler saw the power cap
        sustained = total_ms * 1e-3 >= 1.0 or capped
        key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
        peak = peaks.get(key, 1730.1 if sustained else 1889.9)
        return {"bound": "tensor", "achieved": round(ach, 1), "peak": peak, "unit": "TFLOP/s",
                "frac": round(ach / peak, 4), "traffic": captured_traffic(dom["name"]), "kernel": dom["name"],
                "peak_source": "%s bf16 %s (timed region %.2f s%s)" % (
                    peak_src, "sustained" if sustained else "burst", total_ms * 1e-3,
                    ", power cap seen" if capped else ", no power cap")}
    if dom["name"].startswith("f64_gemm"):
        ach = fl / (avg_ms * 1e-3) / 1e12
        peak = 1.098
        return {"bound": "alu", "achieved": round(ach, 3), "peak": peak, "unit": "TFLOP/s",
                "frac": round(ach / peak, 4), "traffic": None, "kernel": dom["name"],
                "peak_source": "FP64 pipe: cuBLAS DGEMM 4096^3 measured on this GB300 (1.098 TFLOP/s)"}
    ach = by / (avg_ms * 1e-3) / 1e9
    peak = peaks.get("hbm_gbs", 6676.8)
    return {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
            "frac": round(ach / peak, 4), "traffic": None, "kernel": dom["name"],
            "peak_source": "%s hbm" % peak_src}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = max(mx, float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        return dist.get_rank(), ws, local
    return 0, 1, 0


def barrier_max(value, ws):
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda")
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload():
    from paper_2404_19163_gb300 import synth
    return synth.cubic_overlap()


# ------------------------------------------------------------------ CPU oracle timing
def oracle_sample(S, iters):
    """cpu_baseline leg: time one FP64 residual and one polynomial+update of the CPU oracle on the
    full workload (about 17 s on 16 cores) and scale them to the whole Algorithm 2 run, (iters+1)
    residuals + iters updates.  An estimate from a bounded sample, labelled as one."""
    import numpy as np
    import oracle
    n = S.shape[0]
    Z = np.eye(n) * oracle.gershgorin_scale(S)
    t0 = time.perf_counter()
    d, err = oracle.residual(S, Z)
    t1 = time.perf_counter()
    oracle.update(Z, oracle.poly(d, 2))
    t2 = time.perf_counter()
    est_ms = ((iters + 1) * (t1 - t0) + iters * (t2 - t1)) * 1e3
    return est_ms, (t2 - t0), oracle.num_threads()


def oracle_factorization_calls(S, iters, refine_steps=1):
    """The oracle's factorization of S as its sequence of calls (Algorithm 2 with `iters` updates,
    then Algorithm 3's refinement updates, each update followed by its residual): a generator of
    zero-argument callables, each one oracle call on the full workload, run in order."""
    import numpy as np
    import oracle
    n = S.shape[0]
    state = {"Z": np.eye(n) * oracle.gershgorin_scale(S)}

    def residual():
        state["d"], state["err"] = oracle.residual(S, state["Z"])

    def poly():
        state["Q"] = oracle.poly(state["d"], 2)

    def update():
        state["Z"] = oracle.update(state["Z"], state["Q"])

    yield residual
    for _ in range(iters + refine_steps):
        yield poly
        yield update
        yield residual


def run_reference(args, rank, ws):
    """The reference arm: the CPU oracle on this machine's host cores.  One step = one oracle call of the
    workload's factorization (a residual, a polynomial or an update at N = 4096, a few seconds each);
    the timed steps run complete factorizations back to back, and the value is the measured time of
    the first complete one (the sum of its calls' times), not an extrapolation.  When --steps is
    smaller than one factorization's call count, the timed region runs the whole factorization
    anyway and reports the calls it ran as its steps."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    oracle.build()
    S = workload()
    cores = oracle.num_threads()
    small = np.ascontiguousarray(S[:512, :512])
    for _ in range(args.warmup):            # warm-up: a small residual (threads, caches, page-in)
        oracle.residual(small, np.eye(512))
    per_fact = 1 + 3 * (FP64_ITERS_WORKLOAD2 + 1)
    steps = max(args.steps, per_fact)
    call_ms, first_ms = [], None
    gen = oracle_factorization_calls(S, FP64_ITERS_WORKLOAD2)
    t_all = time.perf_counter()
    for k in range(steps):
        try:
            f = next(gen)
        except StopIteration:
            gen = oracle_factorization_calls(S, FP64_ITERS_WORKLOAD2)
            f = next(gen)
        t0 = time.perf_counter()
        f()
        call_ms.append((time.perf_counter() - t0) * 1e3)
        if k + 1 == per_fact:
            first_ms = sum(call_ms)
    wall_s = time.perf_counter() - t_all
    v = first_ms
    sample = ("one complete factorization of the N=4096 workload by the C oracle (OpenMP, %d threads): "
              "Gershgorin start, %d Algorithm 2 updates and 1 Algorithm 3 refinement update, each followed by "
              "its FP64 residual (%d oracle calls, measured call by call; one call per step)"
              % (cores, FP64_ITERS_WORKLOAD2, per_fact))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": args.warmup, "ms_per_step": round(sum(call_ms) / steps, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "gaussian_overlap_cubic_N4096_cold_start", "N": 4096, "order": 2,
                   "precision": "fp64 (CPU oracle)", "tol": TOL},
        "timed_region_s": round(wall_s, 2),
        "cpu_baseline": {"value": round(v, 3), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(v, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, ws, local):
    import numpy as np
    import torch
    from paper_2404_19163_gb300 import Context, build as zbuild
    zbuild.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    S_host = workload()
    n = S_host.shape[0]
    S = torch.from_numpy(S_host).to(dev)
    Z = torch.empty_like(S)
    stream = torch.cuda.Stream(device=dev)
    ctx = Context(local, stream=stream)
    l2_flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    prec = args.precision
    kw = dict(order=2, precision=prec, tol=TOL, Z=Z)
    if args.refine_mode:
        kw["refine_mode"] = args.refine_mode

    # FP64 GPU path on the same input (comparator; untimed here, timed once below)
    r64 = ctx.refine(S, None, order=2, precision="fp64", Z=Z)
    fp64_iters = r64.info["iters"]
    fp64_resid = r64.info["resid_f"] / math.sqrt(n)
    Z64 = Z.clone()

    for _ in range(args.warmup):
        ctx.refine(S, None, **kw)
    torch.cuda.synchronize()

    ctx.set_profiling(True)
    ctx.kernel_stats(reset=True)
    times, launches, infos = [], 0, []
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            l2_flush.zero_()          # outside the timed region: L2 flushed between steps
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = ctx.refine(S, None, **kw)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            launches += r.info["launches"]
            infos.append(r.info)
    torch.cuda.synchronize()
    stats = ctx.kernel_stats(reset=True)
    ctx.set_profiling(False)
    total = barrier_max(sum(times), ws)
    ms = total / args.steps
    value = total / (args.steps * ws)

    # accuracy of the mixed result against the FP64 path
    Zh = Z.cpu().numpy()
    Zr = Z64.cpu().numpy()
    rel_z = float(np.linalg.norm(Zh - Zr) / np.linalg.norm(Zr))
    resid = infos[-1]["resid_f"] / math.sqrt(n)

    # FP64 GPU comparator, timed once (same input, same stop rule)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.refine(S, None, order=2, precision="fp64", Z=Z64)
    e1.record(stream)
    e1.synchronize()
    fp64_ms = e0.elapsed_time(e1)

    # FP32 CUDA-core path ("single") on the same input: bulk to the Algorithm 2 stop + the
    # FP64-accurate residual of its result (it cannot reach tol without refinement)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r32 = ctx.refine(S, None, order=2, precision="fp32", Z=Z64)
    e1.record(stream)
    e1.synchronize()
    fp32_ms = e0.elapsed_time(e1)
    fp32_info = {"ms": round(fp32_ms, 3), "iters": r32.info["iters"], "resid": r32.info["resid_f"] / math.sqrt(n)}
    e0.record(stream)
    r32r = ctx.refine(S, None, order=2, precision="fp32", refine_steps=3, tol=TOL, Z=Z64)
    e1.record(stream)
    e1.synchronize()
    fp32_info.update({"refined_ms": round(e0.elapsed_time(e1), 3), "refined_resid": r32r.info["resid_f"] / math.sqrt(n),
                      "refined_iters": r32r.info["refine_iters"]})

    # the same factorization with the FP64-accurate products by error-free slicing (the fallback
    # scheme) instead of CRT residues: one warm-up, then the best of two
    rm = {"refine_mode": args.refine_mode} if args.refine_mode else {}
    try:
        ctx.set_emulation("slices")
        ctx.refine(S, None, order=2, precision=prec, tol=TOL, Z=Z64, **rm)
        sl_ms = []
        for _ in range(2):
            e0.record(stream)
            rs = ctx.refine(S, None, order=2, precision=prec, tol=TOL, Z=Z64, **rm)
            e1.record(stream)
            e1.synchronize()
            sl_ms.append(e0.elapsed_time(e1))
        slices_info = {"ms": round(min(sl_ms), 3), "resid": rs.info["resid_f"] / math.sqrt(n),
                       "refine_iters": rs.info["refine_iters"]}
    except Exception as e:  # noqa: BLE001 -- a comparator must not cost the bench line
        slices_info = {"unavailable": str(e).splitlines()[0][:200] if str(e) else type(e).__name__}
    finally:
        try:
            ctx.set_emulation("auto")
        except Exception:  # noqa: BLE001
            pass

    # diagonalization comparator (cuSOLVER), once warm: time and the residual of its S^{-1/2}
    try:
        eigh_inverse_sqrt(S)
        Ze, eigh_ms = eigh_inverse_sqrt(S)
        eigh_info = {"ms": round(eigh_ms, 3), "resid": ctx.residual(S, Ze.contiguous(), "ozaki") / math.sqrt(n),
                     "how": "torch.linalg.eigh (cuSOLVER syevd, FP64) + V diag(lambda^-1/2) V^T (cuBLAS)"}
        del Ze
    except RuntimeError as e:  # e.g. torch's linalg library cannot be loaded (seen under a profiler)
        eigh_info = {"unavailable": str(e).splitlines()[0][:200]}

    # e2e: host (pinned) buffers through the public C ABI, copies inside the call
    S_pin = torch.from_numpy(S_host).pin_memory()
    Z_pin = torch.empty_like(S_pin).pin_memory()
    e2e = []
    for _ in range(max(3, min(args.steps, 7))):  # the median of several, against host noise
        t0 = time.perf_counter()
        ctx.refine(S_pin, None, order=2, precision=prec, tol=TOL, Z=Z_pin,
                   **({"refine_mode": args.refine_mode} if args.refine_mode else {}))
        e2e.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = barrier_max(statistics.median(e2e), ws)

    # roofline of the dominant kernel family
    peaks, peak_src = measured_peaks()
    dom = max(stats, key=lambda s: s["ms"]) if stats else None
    roof = None
    if dom:
        roof = roofline_of(dom, total, clk.summary()["reasons"], peaks, peak_src)
    tc_ms = sum(s["ms"] for s in stats if s["name"].startswith("tc_gemm"))
    tc_fl = sum(s["flops"] for s in stats if s["name"].startswith("tc_gemm"))
    # the FP64-accurate products counted as the FP64 products they stand for (2 N^2 K each, half on
    # symmetric tiles), over the time of everything that forms them (residues, products, reconstruction)
    emu_fl = sum(s["flops"] for s in stats if s["name"] == "fp64_equiv")
    emu_ms = sum(s["ms"] for s in stats if s["name"] in ("tc_gemm.crt", "oz_crt", "oz_residues", "tc_gemm.ozaki",
                                                          "oz_combine", "oz_slice", "oz_crt.wide",
                                                          "oz_residues.wide"))
    fp64_equiv = {"flops_per_step": emu_fl / args.steps, "ms_per_step": round(emu_ms / args.steps, 3),
                  "tflops": round(emu_fl / (emu_ms * 1e-3) / 1e12, 1) if emu_ms > 0 else None,
                  "executed_tensor_tflops_same_kernels": round(
                      sum(s["flops"] for s in stats if s["name"] in ("tc_gemm.crt", "tc_gemm.ozaki")) /
                      (emu_ms * 1e-3) / 1e12, 1) if emu_ms > 0 else None}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        est, secs, cores = oracle_sample(S_host, fp64_iters)
        cpu = {"value": round(est, 1), "unit": UNIT, "cores": cores, "kind": "oracle", "estimate": True,
               "sample": ("bounded sample: one FP64 residual + one polynomial/update of the C oracle at N=4096 "
                          "(%.1f s measured), scaled to the %d-update Algorithm 2 run; the reference arm "
                          "measures a complete factorization" % (secs, fp64_iters))}

    ctx.close()
    extras = {}
    if rank == 0 and ws == 1 and not args.no_extras:
        # workloads 3 and 4 beside the headline, each with the FP64 GPU path on the same inputs
        del S, Z, Z64, l2_flush
        torch.cuda.empty_cache()
        for key, leg in (("ill", lambda: ill_leg(args, steps=2, fp64_comparator=True)),
                         ("batched", lambda: batched_leg(args, 0, 1, local, frames_timed=2, fp64_comparator=True))):
            try:
                extras[key] = leg()
            except Exception as e:  # noqa: BLE001 -- an extra leg must not cost the headline line
                extras[key] = {"unavailable": (str(e).splitlines() or [type(e).__name__])[0][:300]}
            torch.cuda.empty_cache()

    if rank == 0:
        out = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16" if prec.startswith("bf16") else ("fp16" if prec.startswith("fp16") else prec), "data": "synthetic",
            "config": {"workload": "gaussian_overlap_cubic_N4096_cold_start", "N": n, "order": 2,
                       "precision": prec, "refine": "Algorithm 3, FP64 d (%s)" % (args.refine_mode or "default"),
                       "tol": TOL, "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "flushed between timed steps (256 MiB write); S alone is 134 MB > L2"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": round(e2e_ms, 3), "unit": UNIT, "h2d_bytes_per_step": n * n * 8,
                    "d2h_bytes_per_step": n * n * 8 + 8 * 128},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "iters": infos[-1]["iters"], "refine_iters": infos[-1]["refine_iters"],
            "resid": resid, "rel_z_vs_fp64": rel_z,
            "fp64_path": {"ms": round(fp64_ms, 3), "iters": fp64_iters, "resid": fp64_resid},
            "fp32_path": fp32_info,
            "slices_path": slices_info,
            "speedup_vs_slices": round(slices_info["ms"] / ms, 2) if "ms" in slices_info else None,
            "eigh_comparator": eigh_info,
            "speedup_vs_fp64_path": round(fp64_ms / ms, 2),
            "speedup_vs_eigh": round(eigh_info["ms"] / ms, 2) if "ms" in eigh_info else None,
            "tc_tflops": round(tc_fl / (tc_ms * 1e-3) / 1e12, 1) if tc_ms > 0 else None,
            "fp64_equiv": fp64_equiv,
            "kernels": sorted([{k: (round(v, 4) if isinstance(v, float) else v) for k, v in s.items()}
                               for s in stats], key=lambda s: -s["ms"]),
        }
        out.update(extras)
        print(json.dumps(out), flush=True)


def eigh_inverse_sqrt(S):
    """Comparator (the paper's diagonalization route, Sec. 2 and Sec. 5.1): S^{-1/2} =
    V diag(lambda^{-1/2}) V^T with torch.linalg.eigh (cuSOLVER) and one cuBLAS product, timed
    with CUDA events on torch's current stream.  Returns (Z, ms)."""
    import torch
    st = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    lam, V = torch.linalg.eigh(S)
    Z = (V * lam.rsqrt()) @ V.T
    e1.record(st)
    e1.synchronize()
    return Z, e0.elapsed_time(e1)


def run_case_residual(args):
    """Profiling case: the FP64-accurate residual d = I - Z^T S Z (error-free slicing on
    the tensor cores) of workload 2 at a converged Z; prints its own JSON line."""
    import numpy as np
    import torch
    from paper_2404_19163_gb300 import Context, build as zbuild
    zbuild.build()
    S = torch.from_numpy(workload()).cuda()
    n = S.shape[0]
    with Context(0) as ctx:
        Z = ctx.refine(S, None, order=2, precision="fp64").Z   # CUDA-core kernels only: the
        # first tensor-core launches below are the two sliced products of the residual
        D = torch.empty_like(S)
        for _ in range(args.warmup):
            ctx.residual(S, Z, "ozaki", D=D)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            err = ctx.residual(S, Z, "ozaki", D=D)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / args.steps
    print(json.dumps({"case": "residual_ozaki", "N": n, "ms": round(ms, 3), "err": err}), flush=True)


def run_case_learn(args):
    """Profiling case: the learned start's kernels alone.  The 16 features of workload 2's S
    (row statistics, d0, E^2 on the tensor cores, traces) W + K times, then W + K full-batch
    training steps (forward/backward and Adam) of the 16-64-64-5 network on 20 000 feature rows
    drawn from a seeded normal; prints its own JSON line."""
    import numpy as np
    import torch
    from paper_2404_19163_gb300 import Context, learn, build as zbuild
    zbuild.build()
    S = torch.from_numpy(workload()).cuda()
    g = np.random.default_rng(7)
    rows = 20000
    X = torch.from_numpy(g.standard_normal((rows, 16)).astype(np.float32)).cuda()
    ts = torch.from_numpy(g.uniform(0.5, 1.5, rows).astype(np.float32)).cuda()
    to = torch.from_numpy(g.integers(0, 4, rows).astype(np.int32)).cuda()
    with Context(0) as ctx:
        P = torch.from_numpy(learn.init_params(0)).cuda()
        M, V = torch.zeros_like(P), torch.zeros_like(P)
        mu, sd = X.mean(0), X.std(0) + 1e-6
        for _ in range(args.warmup):
            ctx.features(S)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            f = ctx.features(S)
        torch.cuda.synchronize()
        ms_feat = (time.perf_counter() - t0) * 1e3 / args.steps
        for step in range(1, args.warmup + 1):
            grad, loss = ctx.mlp_backward(P, mu, sd, X, ts, to, 1.0)
            ctx.mlp_adam(P, grad, M, V, step)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for step in range(args.warmup + 1, args.warmup + args.steps + 1):
            grad, loss = ctx.mlp_backward(P, mu, sd, X, ts, to, 1.0)
            ctx.mlp_adam(P, grad, M, V, step)
        torch.cuda.synchronize()
        ms_train = (time.perf_counter() - t0) * 1e3 / args.steps
    print(json.dumps({"case": "learn", "N": int(S.shape[0]), "features_ms": round(ms_feat, 3),
                      "train_step_ms": round(ms_train, 3), "rows": rows, "loss": loss,
                      "features": [float(x) for x in f]}), flush=True)


def batched_leg(args, rank=0, ws=1, local=0, frames_timed=None, fp64_comparator=False):
    """Workload 4: 128 cluster overlaps, N_i ~ U[256, 3072], frames of a trajectory (sites
    displaced by N(0, 0.02^2) per frame); frame 0 is a cold start (untimed), the next frames are
    warm-started from the previous frame's Z and timed with CUDA events, one zfact_refine_batched
    call each.  With several ranks the instances are sharded (greedy by N^3, no data-path
    collective); the frame time is the maximum over ranks (strong scaling: the batch is fixed).
    fp64_comparator: the FP64 GPU path (CUDA-core FP64, Algorithm 2's stop) on the last timed
    frame's matrices from the same warm starts, one instance after another.  Returns a dict."""
    import numpy as np
    import torch
    from paper_2404_19163_gb300 import Context, synth, shard, build as zbuild
    zbuild.build()
    count = args.batch_count
    all_sizes, frame = synth.trajectory(count=count)
    mine = shard.mine(list(all_sizes), rank, ws) if ws > 1 else list(range(count))
    sizes = [int(all_sizes[i]) for i in mine]
    frames = 1 + max(1, frames_timed if frames_timed else args.steps)
    stream = torch.cuda.Stream()
    ctx = Context(local, stream=stream)
    prec = args.precision

    def mats(f):
        pos = frame.positions(f)
        return [synth.gaussian_overlap_torch(pos[i]) for i in mine]

    S0 = mats(0)
    Zp, h, infos, st = ctx.refine_batched(S0, None, precision=prec)
    cold_iters = [i["iters"] for i in infos]
    del S0
    times, iters, resid, launches = [], [], [], 0
    ctx.set_profiling(True)
    ctx.kernel_stats(reset=True)
    Zprev, Sf = Zp, None
    with ClockSampler(local) as clk:
        for f in range(1, frames):
            Sf = mats(f)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            Zf, h, infos, st = ctx.refine_batched(Sf, Zp, precision=prec)
            e1.record(stream)
            e1.synchronize()
            times.append(barrier_max(e0.elapsed_time(e1), ws))
            iters.append([i["iters"] for i in infos])
            resid.append(max(i["resid_f"] / math.sqrt(n) for i, n in zip(infos, sizes)))
            launches += infos[0]["launches"]
            Zprev, Zp = Zp, Zf
    stats = ctx.kernel_stats(reset=True)
    ctx.set_profiling(False)
    fp64 = None
    if fp64_comparator:
        # the same frame (Sf) from the same warm starts (Zprev) through the FP64 GPU path
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        outs = [torch.empty_like(S) for S in Sf]
        torch.cuda.synchronize()
        e0.record(stream)
        it64, r64 = [], []
        for S, Z0, Zo in zip(Sf, Zprev, outs):
            r = ctx.refine(S, Z0, order=2, precision="fp64", Z=Zo, raise_on_error=False)
            it64.append(r.info["iters"])
            r64.append(r.info["resid_f"] / math.sqrt(S.shape[0]))
        e1.record(stream)
        e1.synchronize()
        ms64 = barrier_max(e0.elapsed_time(e1), ws)
        fp64 = {"ms": round(ms64, 2), "iters_mean": float(np.mean(it64)), "max_resid_over_sqrtN": max(r64),
                "how": "zfact_refine precision fp64 (CUDA-core FP64 products, Algorithm 2 stop), instance by "
                       "instance from the same warm starts"}
    ctx.close()
    tc = [k for k in stats if k["name"].startswith("tc_gemm.b_")]
    tc_ms = sum(k["ms"] for k in tc)
    tc_fl = sum(k["flops"] for k in tc)
    sum_n3 = float(np.sum(np.asarray(all_sizes, dtype=np.float64) ** 3))
    frame_ms = statistics.mean(times)
    bulk_ms = sum(k["ms"] for k in stats if k["name"].startswith("tc_gemm.b_") or k["name"].startswith("b_")) / len(times)
    out = {
        "workload": "batched_trajectory_128_clusters_N256-3072_warm_frames",
        "metric": "ms per frame (all 128 factorizations, bulk + FP64-accurate final residual)",
        "value": round(frame_ms, 3), "unit": "ms", "frames_timed": len(times),
        "n_gpus": ws, "scaling": "strong", "higher_is_better": False,
        "precision": prec, "sum_N": int(np.sum(all_sizes)), "sum_N3": sum_n3,
        "cold_iters_mean": float(np.mean(cold_iters)),
        "warm_iters_mean": float(np.mean(iters)), "warm_iters_max": int(np.max(iters)),
        "max_resid_over_sqrtN": max(resid), "gpu_launches": launches,
        "grouped_tc_tflops": round(tc_fl / (tc_ms * 1e-3) / 1e12, 1) if tc_ms else None,
        "grouped_bulk_ms_per_frame": round(bulk_ms, 2),
        "clocks": clk.summary(),
        "kernels": sorted([{k: (round(v, 3) if isinstance(v, float) else v) for k, v in x.items()}
                           for x in stats], key=lambda x: -x["ms"])[:10],
    }
    if fp64:
        out["fp64_path"] = fp64
        out["speedup_vs_fp64_path"] = round(fp64["ms"] / frame_ms, 2)
    return out if rank == 0 else None


def run_case_factor(args):
    """Profiling case: the headline factorization alone (workload 2, the benchmark's precision and
    refinement), W warm-up and K timed calls and nothing else, so that a launch list of it holds only
    factorizations; prints its own JSON line with the launches per factorization."""
    import torch
    from paper_2404_19163_gb300 import Context, build as zbuild
    zbuild.build()
    S = torch.from_numpy(workload()).cuda()
    n = S.shape[0]
    Z = torch.empty_like(S)
    with Context(0) as ctx:
        kw = dict(order=2, precision=args.precision, tol=TOL, Z=Z)
        for _ in range(args.warmup):
            r = ctx.refine(S, None, **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            r = ctx.refine(S, None, **kw)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / args.steps
    print(json.dumps({"case": "factor", "N": n, "ms": round(ms, 3), "launches_per_factorization": r.info["launches"],
                      "resid": r.info["resid_f"] / math.sqrt(n)}), flush=True)


def run_batched(args, rank=0, ws=1, local=0):
    out = batched_leg(args, rank, ws, local, fp64_comparator=args.fp64_comparator)
    if out is not None:
        print(json.dumps(out), flush=True)


def ill_leg(args, steps=None, fp64_comparator=False, cond=False, eigh=False):
    """Workload 3: fcc Gaussian overlap, 4 exponents per site, N = 16384 (cond ~1e5-1e6),
    warm start Z0 = the converged factor of the same system with sites displaced by
    N(0, 0.01^2); FP16 hi/lo split bulk, Algorithm 3 refinement with FP64-accurate d, to
    ||I - Z^T S Z||_F / sqrt(N) <= tol.  Timed with CUDA events on the context's stream; the FP64
    GPU path from the same warm start once when fp64_comparator.  Returns a dict."""
    import torch
    from paper_2404_19163_gb300 import Context, synth, build as zbuild
    zbuild.build()
    S = synth.fcc_overlap_torch()
    n = S.shape[0]
    cond_v = None
    if cond:
        lam = torch.linalg.eigvalsh(S)
        cond_v = float(lam[-1] / lam[0])
        del lam
    Sp = synth.fcc_overlap_torch(perturb=0.01)
    stream = torch.cuda.Stream()
    ctx = Context(0, stream=stream)
    prec = "fp16_split" if args.precision == "bf16_split" else args.precision
    Z0 = ctx.refine(Sp, None, order=2, precision=prec, tol=0.0, raise_on_error=False).Z
    del Sp
    Z = torch.empty_like(S)
    kw = dict(order=2, precision=prec, tol=args.tol_ill, Z=Z, raise_on_error=False)
    r = ctx.refine(S, Z0, **kw)  # warm-up
    ctx.set_profiling(True)
    ctx.kernel_stats(reset=True)
    times, infos = [], []
    with ClockSampler(0) as clk:
        for _ in range(steps or args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = ctx.refine(S, Z0, **kw)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            infos.append(dict(r.info, status=r.status))
    stats = ctx.kernel_stats(reset=True)
    ctx.set_profiling(False)
    out = {"workload": "fcc_overlap_N16384_4exp_warm_start", "metric": METRIC, "value": round(statistics.mean(times), 2),
           "unit": "ms", "steps": len(times), "N": n, "precision": prec, "tol": args.tol_ill,
           "iters": infos[-1]["iters"], "refine_iters": infos[-1]["refine_iters"], "status": infos[-1]["status"],
           "resid": infos[-1]["resid_f"] / math.sqrt(n),
           "hist": [float(h) for h in r.hist], "clocks": clk.summary(),
           "kernels": sorted([{k: (round(v, 3) if isinstance(v, float) else v) for k, v in x.items()}
                              for x in stats], key=lambda x: -x["ms"])[:8]}
    if cond_v is not None:
        out["cond"] = cond_v
    if fp64_comparator:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r64 = ctx.refine(S, Z0, order=2, precision="fp64", Z=Z, raise_on_error=False)
        e1.record(stream)
        e1.synchronize()
        out["fp64_path"] = {"ms": round(e0.elapsed_time(e1), 1), "iters": r64.info["iters"],
                            "resid": r64.info["resid_f"] / math.sqrt(n), "hist": [float(h) for h in r64.hist]}
        out["speedup_vs_fp64_path"] = round(out["fp64_path"]["ms"] / out["value"], 2)
    if eigh:
        try:
            with torch.cuda.stream(stream):
                eigh_inverse_sqrt(S[:256, :256].contiguous())  # warm the solver
                Ze, eigh_ms = eigh_inverse_sqrt(S)
            out["eigh_comparator"] = {"ms": round(eigh_ms, 1),
                                      "resid": ctx.residual(S, Ze.contiguous(), "ozaki") / math.sqrt(n)}
            del Ze
        except RuntimeError as e:
            out["eigh_comparator"] = {"unavailable": str(e).splitlines()[0][:200]}
    ctx.close()
    return out


def run_ill(args):
    out = ill_leg(args, fp64_comparator=args.fp64_comparator, cond=True, eigh=args.fp64_comparator)
    print(json.dumps(out), flush=True)


def run_paper(args):
    """The paper's synthetic overlap (Sec. 5.1): S = (T + T^T)/2 shifted to lambda_min = 0.5,
    Z0 = S^{-1/2} + 0.005 U.  For every N, each method of Table I that the library offers runs from
    that Z0 under Algorithm 2's stop (Fig. 2): the (h)(h)+(h)(l)+(l)(h) split with and without the
    FP64-accurate refinement, (h)(h) with and without a single-precision refinement step, (h)(h)half
    (FP16 accumulation), single, and double (N <= 4096).  Per method: iterations, the Frobenius history, the stop ratios
    Err_n / Err_{n-1}^3 (Fig. 1, Fig. 2 top), the FP64-accurate residual of the result and the time
    (Fig. 3), with cuSOLVER's eigh as the diagonalization comparator.  One JSON line."""
    import torch
    from paper_2404_19163_gb300 import Context, synth, build as zbuild
    zbuild.build()
    stream = torch.cuda.Stream()
    ctx = Context(0, stream=stream)
    methods = [("split+refi", dict(precision="fp16_split", tol=TOL)),
               ("split", dict(precision="fp16_split", refine_steps=0)),
               ("hh+refi_fp32", dict(precision="fp16", refine_mode="fp32", refine_steps=1)),
               ("hh", dict(precision="fp16", refine_steps=0)),
               ("hh_half", dict(precision="fp16_half", refine_steps=0)),
               ("single", dict(precision="fp32")),
               ("double", dict(precision="fp64"))]
    rows = []
    for n in [int(x) for x in args.paper_sizes.split(",")]:
        S = synth.paper_synthetic_torch(n)
        Z0 = synth.paper_start_torch(S, 0.005, seed=0)
        Z = torch.empty_like(S)
        row = {"N": n, "methods": {}}
        for name, kw in methods:
            if name == "double" and n > 4096:
                continue
            kw = dict(order=2, Z=Z, raise_on_error=False, **kw)
            ctx.refine(S, Z0, **kw)  # warm-up
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = ctx.refine(S, Z0, **kw)
            e1.record(stream)
            e1.synchronize()
            h = [float(x) for x in r.hist]
            it = r.info["iters"]
            row["methods"][name] = {
                "iters": it, "refine_iters": r.info["refine_iters"], "status": r.status,
                "ms": round(e0.elapsed_time(e1), 3), "resid": r.info["resid_f"] / math.sqrt(n), "hist": h,
                "stop_ratios": [h[i] / h[i - 1] ** 3 for i in range(1, it + 1)]}
        try:
            with torch.cuda.stream(stream):
                Ze, eigh_ms = eigh_inverse_sqrt(S)
            row["eigh_ms"] = round(eigh_ms, 2)
            row["eigh_resid"] = ctx.residual(S, Ze.contiguous(), "ozaki") / math.sqrt(n)
            del Ze
        except RuntimeError as e:
            row["eigh_unavailable"] = str(e).splitlines()[0][:200]
        del S, Z0, Z
        torch.cuda.empty_cache()
        rows.append(row)
        print(json.dumps({"N": n, **{k: (v["iters"], v["ms"], v["resid"]) for k, v in row["methods"].items()},
                          "eigh_ms": row.get("eigh_ms")}), file=sys.stderr, flush=True)
    ctx.close()
    print(json.dumps({"workload": "paper_synthetic_sweep", "alpha": 0.005, "gamma": 0.5, "tol": TOL,
                      "rows": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16_split")
    ap.add_argument("--refine-mode", default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the workload 3 and 4 legs that the default line carries as extra keys")
    ap.add_argument("--case", default=None, choices=[None, "residual", "factor", "learn"])
    ap.add_argument("--workload", default="single", choices=["single", "batched", "ill", "paper"])
    ap.add_argument("--paper-sizes", default="1024,4096,16384")
    ap.add_argument("--tol-ill", type=float, default=1e-12)
    ap.add_argument("--fp64-comparator", action="store_true")
    ap.add_argument("--batch-count", type=int, default=128)
    args = ap.parse_args()
    if args.case == "residual":
        run_case_residual(args)
        return
    if args.case == "factor":
        run_case_factor(args)
        return
    if args.case == "learn":
        run_case_learn(args)
        return
    if args.workload == "batched":
        rank, ws, local = dist_setup()
        run_batched(args, rank, ws, local)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    if args.workload == "ill":
        run_ill(args)
        return
    if args.workload == "paper":
        run_paper(args)
        return
    args.warmup = max(args.warmup, 1)
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        run_reference(args, rank, int(os.environ.get("WORLD_SIZE", "1")))
        return
    rank, ws, local = dist_setup()
    run_ours(args, rank, ws, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
