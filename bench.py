"""Benchmark of the nnCANDELINC hot path (Alg. 1) on one GB300.

A step is one whole Alg. 1 run on one synthetic problem: nnTD of X (all its
sweeps, with the per-sweep FP64 relative-error trace), nnCP of the core, the
lift A^(n) = F^(n) B^(n) and the final one-pass residual of the lifted model.
Every step restarts from the same initial factors. The value is nnTD sweeps
per second over the timed steps (device time, inputs resident in HBM).

The default workload is the 512^3 precision workload under the paper's
protocol (5000 iterations per sub-solve, Sec. 4.1): the nnTD sweeps run on the
BF16 copy of X except the last 200, which are FP32 (TF32x3) refinement sweeps.
The same step with FP32 passes throughout is timed beside it, and both final
relative errors come from explicit FP64 passes: the comparison at equal
relative error. Convergence records (exact checkpoints every 50 sweeps) give
the sweeps and time each path needs to reach stated errors.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--impl native|reference]

--impl reference times the FP64 CPU oracle (the only reference this project
has) on the host cores, one bounded sample of the same workload per step.
Under torchrun (N > 1) every rank runs an independent replica (weak scaling,
no data-path collective); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
# The batching form runs up to 8 concurrent fits of three streams each: give the
# process enough hardware work queues (before CUDA starts) so that they do not
# share queues and serialise.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "cp16_512x512x512_m32_bf16_5000"
METRIC = "nnCANDELINC iters/s & TTM TFLOP/s (% roofline), BF16 vs FP32 at equal rel-error"
L2_FLUSH_BYTES = 512 << 20
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--workload", default=DEFAULT_WORKLOAD)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-precision-form", action="store_true")
    p.add_argument("--no-differentiation-form", action="store_true")
    p.add_argument("--no-batching-form", action="store_true")
    p.add_argument("--no-4way-ntd", action="store_true")
    p.add_argument("--no-paper-batch", action="store_true")
    p.add_argument("--no-multirank-study", action="store_true")
    p.add_argument("--no-convergence", action="store_true")
    p.add_argument("--no-256cube", action="store_true")
    return p.parse_args()


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "native" else "gloo"
        dist.init_process_group(backend)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world, device=None):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as fh:
                return json.load(fh), "measured"
        except Exception:
            pass
    return dict(FALLBACK_PEAKS), "fallback"


def peak_value(peaks, *keys):
    for k in keys:
        v = peaks.get(k)
        if isinstance(v, (int, float)):
            return float(v)
        if isinstance(v, dict):
            for kk in ("value", "gbs", "tflops"):
                if isinstance(v.get(kk), (int, float)):
                    return float(v[kk])
    return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def stored_traffic(kernel_name, source_files):
    """DRAM bytes per launch of `kernel_name` from the committed ncu summary, if
    the kernel's sources are unchanged since the capture; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        with open(path) as fh:
            rec = json.load(fh).get(kernel_name)
    except Exception:
        return None
    if not rec:
        return None
    h = hashlib.sha256()
    for f in source_files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    if rec.get("source_sha256") != h.hexdigest():
        return None
    return rec.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------

def _precision_of(w):
    import torch
    if w.dtype == "bf16":
        return "bf16", torch.float32, "bf16"
    if w.dtype == "f64":
        return "fp64", torch.float64, "f64"
    return "fp32", torch.float32, "f32"


class Alg1Step:
    """One whole Alg. 1 run on resident inputs: nnTD of X (every sweep, with
    the FP64 trace), nnCP of the core, the lift and the lifted residual; every
    step restarts from the same initial factors."""

    def __init__(self, w, X, F0d, G0d, B0d, precision, refine_iters, exact_every=0,
                 refine_tol=0.0):
        self.w, self.X, self.F0d, self.G0d, self.B0d = w, X, F0d, G0d, B0d
        self.precision, self.refine = precision, refine_iters
        self.exact_every, self.refine_tol = exact_every, refine_tol
        self.F = [f.clone() for f in F0d]
        self.G = G0d.clone()
        self.B = [b.clone() for b in B0d]
        self.out = {}

    def __call__(self):
        from paper_1909_07570_gb300 import native
        for a, b in zip(self.F, self.F0d):
            a.copy_(b)
        self.G.copy_(self.G0d)
        for a, b in zip(self.B, self.B0d):
            a.copy_(b)
        _, tr = native.ntd_fit(self.X, self.F, self.G, self.w.iters, precision=self.precision,
                               refine_iters=self.refine, trace=True, rel_err=False,
                               exact_every=self.exact_every, refine_tol=self.refine_tol)
        if self.precision == "bf16":
            self.out["refine_from"] = native.nnc_last_refine_sweep()
        native.nncp_core_fit(self.G, self.B, self.w.cp_iters, precision=self.precision,
                             rel_err=False)
        A = native.candelinc_lift(self.F, self.B)
        rn, xn = native.recon_residual(self.X, A)
        self.out["trace"] = tr
        self.out["lifted_rel_err"] = rn / xn
        return tr

    def tucker_rel_err(self):
        from paper_1909_07570_gb300 import native
        rn, xn = native.recon_residual(self.X, self.F, self.G)
        return rn / xn


def timed_steps(step, n, flush, stream):
    """Device time (ms) of n steps, each bracketed by CUDA events on the
    launching stream, an L2 flush (a write larger than L2) before each."""
    import torch
    ms = []
    for _ in range(n):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms


def pass_rooflines(prof, w, dt_bytes, peaks, peak_src, workload):
    """Roofline records of the passes over X from the event profiler's totals:
    one per pass kind that ran, the dominant (largest total time) first."""
    import numpy as np

    from paper_1909_07570_gb300 import native
    hbm = peak_value(peaks, "hbm_gbs", "hbm_GBps", "hbm") or FALLBACK_PEAKS["hbm_gbs"]
    nX = int(np.prod(w.dims))
    names = {0: "ttm_rows_kernel", 1: "ttm_cols_kernel", 2: "tc_pass_kernel<bf16> (X x_3 F3^T)",
             3: "tc_pass_kernel<bf16> (X x_1 F1^T)", 4: "tc_pass_kernel<tf32x3> (X x_3 F3^T)",
             5: "tc_pass_kernel<tf32x3> (X x_1 F1^T)"}
    recs = []
    for kind in sorted(prof, key=lambda k: prof[k][1], reverse=True):
        n_l, ms_l = prof[kind]
        if not n_l:
            continue
        avg_s = (ms_l / n_l) / 1e3
        elem = 2 if kind in (2, 3) else dt_bytes  # the BF16 copy of X, else X itself
        alg_bytes = nX * elem
        alg_flops = 2.0 * nX * (w.m[2] if kind % 2 == 0 else w.m[0])
        achieved = alg_bytes / avg_s / 1e9
        sources = ["paper_1909_07570_gb300/csrc/ttm.cu"] if kind in (0, 1) else \
            ["paper_1909_07570_gb300/csrc/tc_ttm.cu", "paper_1909_07570_gb300/csrc/mma32.cuh"]
        recs.append({
            "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4),
            "traffic": stored_traffic(f"{native.PASS_KINDS[kind]}:{workload}", sources),
            "kernel": names[kind], "pass": native.PASS_KINDS[kind], "launches": n_l,
            "avg_launch_us": round(avg_s * 1e6, 3), "algorithmic_bytes_per_launch": alg_bytes,
            "flops_per_launch": alg_flops, "achieved_tflops": round(alg_flops / avg_s / 1e12, 3),
            "peak_source": f"{peak_src} ({'of measured' if peak_src == 'measured' else 'of fallback'})",
            "timing": "CUDA events around the pass in every 16th sweep of a separate profiled "
                      "run (not the timed steps), on the private stream that launches it",
        })
    return recs


def sweeps_to_target(trace, target):
    """First sweep (1-based) whose trace entry is <= target, else None."""
    import numpy as np
    hit = np.nonzero(np.asarray(trace) <= target)[0]
    return int(hit[0]) + 1 if hit.size else None


def run_native(args, rank, world):
    import numpy as np
    import torch

    from paper_1909_07570_gb300 import inputs, native

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = inputs.WORKLOADS[args.workload]
    precision, dt, dname = _precision_of(w)
    X64, _, F0, G0, B0 = inputs.make_problem(
        inputs.Workload(**{**w.__dict__, "seed": w.seed + 17 * rank}))
    Xh = torch.tensor(X64, dtype=dt).pin_memory()
    X = Xh.to(dev)
    F0d = [torch.tensor(f, dtype=dt, device=dev) for f in F0]
    G0d = torch.tensor(G0, dtype=dt, device=dev)
    B0d = [torch.tensor(b, dtype=dt, device=dev) for b in B0]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    step = Alg1Step(w, X, F0d, G0d, B0d, precision, w.refine_iters)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    launches0 = native.nnc_kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    step_ms = timed_steps(step, args.steps, flush, stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    gpu_launches = native.nnc_kernel_launches() - launches0
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    ms_per_step = total_ms / args.steps
    value = world * w.iters * args.steps / (total_ms / 1e3)
    tucker_err = step.tucker_rel_err()
    lifted_err = step.out["lifted_rel_err"]
    trace = step.out["trace"].cpu().numpy()

    result = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "iters/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": dname,
        "data": "synthetic (seeded planted nonnegative CP + uniform noise)",
        "config": {
            "workload": args.workload, "dims": list(w.dims), "m": list(w.m), "r": w.r,
            "planted_rank": w.planted_rank, "ntd_sweeps_per_step": w.iters,
            "nncp_sweeps_per_step": w.cp_iters, "refine_sweeps": w.refine_iters,
            "step": "ntd_fit (with FP64 trace) + nncp_core_fit + candelinc_lift + recon_residual",
            "passes": {"fp32": "tcgen05 TF32x3 (FP32-accurate, 3 products per term)",
                       "bf16": "tcgen05 BF16 with per-slice power-of-two scales; the last "
                               f"{w.refine_iters} sweeps tcgen05 TF32x3 (FP32 refinement)",
                       "fp64": "SIMT FP64"}[precision],
            "l2": f"X ({X.numel() * X.element_size() >> 20} MiB) larger than L2, and flushed "
                  f"between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
            "parallelism": "replicas" if world > 1 else "single GPU",
        },
        "gpu_launches": int(gpu_launches),
        "final_tucker_rel_err": tucker_err,
        "final_tucker_rel_err_trace": float(trace[-1]),
        "final_lifted_rel_err": lifted_err,
        "clocks": clk,
    }
    peaks, peak_src = load_peaks()

    # The same step with the plain FP32 (TF32x3) passes: the comparison at
    # equal relative error (same sweeps, same start; both final errors from an
    # explicit FP64 pass).
    if precision == "bf16" and rank == 0 and world == 1:
        step32 = Alg1Step(w, X, F0d, G0d, B0d, "fp32", 0)
        step32()
        n32 = max(1, min(args.steps, 3))
        ms32 = timed_steps(step32, n32, flush, stream)
        v32 = w.iters * n32 / (sum(ms32) / 1e3)
        e32 = step32.tucker_rel_err()
        result["fp32_comparison"] = {
            "value": round(v32, 3), "unit": "iters/s", "steps": n32,
            "ms_per_step": round(sum(ms32) / n32, 4),
            "final_tucker_rel_err": e32, "final_lifted_rel_err": step32.out["lifted_rel_err"],
            "bf16_speedup": round(value / v32, 3),
            "abs_tucker_rel_err_diff_bf16_vs_fp32": abs(tucker_err - e32),
            "rel_tucker_rel_err_diff_bf16_vs_fp32": abs(tucker_err - e32) / e32,
            # The reduced-precision path's bound against the FP64 oracle.
            "equal_rel_err_bound": 1e-3,
        }

    # Rooflines of the passes over X, from a separate run with the event
    # profiler on (the timed steps above ran without it).
    native.nnc_profile_enable(True)
    step()
    torch.cuda.synchronize()
    prof = {k: native.nnc_profile_read(k) for k in native.PASS_KINDS}
    native.nnc_profile_enable(False)
    recs = pass_rooflines(prof, w, X.element_size(), peaks, peak_src, args.workload)
    result["roofline"] = recs[0] if recs else None
    result["pass_rooflines"] = recs
    nX = int(np.prod(w.dims))
    pass_ms = sum(v[1] for v in prof.values())
    flops_all = sum(prof[k][0] * 2.0 * nX * (w.m[2] if k % 2 == 0 else w.m[0]) for k in prof)
    result["ttm_tflops"] = round(flops_all / (pass_ms / 1e3) / 1e12, 3) if pass_ms else None

    # End to end through the public API with host buffers: H2D of X and the
    # initial factors from pinned memory, the whole step, D2H of the lifted
    # factors and the scalar result, on the device clock of the host (wall).
    F0h = [torch.tensor(f, dtype=dt).pin_memory() for f in F0]
    G0h = torch.tensor(G0, dtype=dt).pin_memory()
    B0h = [torch.tensor(b, dtype=dt).pin_memory() for b in B0]
    A_h = [torch.empty(n, w.r, dtype=dt).pin_memory() for n in w.dims]
    h2d = Xh.numel() * Xh.element_size() + sum(f.numel() * f.element_size() for f in F0h) + \
        G0h.numel() * G0h.element_size() + sum(b.numel() * b.element_size() for b in B0h)
    d2h = sum(a.numel() * a.element_size() for a in A_h) + 8

    def e2e_step():
        Xd = Xh.to(dev, non_blocking=True)
        Fd = [f.to(dev, non_blocking=True) for f in F0h]
        Gd = G0h.to(dev, non_blocking=True)
        Bd = [b.to(dev, non_blocking=True) for b in B0h]
        native.ntd_fit(Xd, Fd, Gd, w.iters, precision=precision, refine_iters=w.refine_iters,
                       trace=True, rel_err=False)
        native.nncp_core_fit(Gd, Bd, w.cp_iters, precision=precision, rel_err=False)
        A = native.candelinc_lift(Fd, Bd)
        rn, xn = native.recon_residual(Xd, A)
        for a, ah in zip(A, A_h):
            ah.copy_(a, non_blocking=True)
        torch.cuda.synchronize()
        return rn / xn

    e2e_step()
    n_e2e = max(1, min(args.steps, 5))
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    result["e2e"] = {"value": round(world * w.iters * n_e2e / e2e_s, 3), "unit": "iters/s",
                     "steps": n_e2e, "h2d_bytes_per_step": int(h2d),
                     "d2h_bytes_per_step": int(d2h)}

    # Convergence at equal relative error: exact checkpoints every 50 sweeps
    # (explicit FP64 passes) for both paths; sweeps and device time to reach
    # stated relative errors, with the per-sweep times of the timed steps.
    if precision == "bf16" and rank == 0 and world == 1 and not args.no_convergence:
        result["convergence"] = convergence(w, X, F0d, G0d, B0d, value, result)
    return result, (X64, F0, G0, w)


def convergence(w, X, F0d, G0d, B0d, value_bf16, result):
    import torch

    from paper_1909_07570_gb300 import native
    every = 50
    out = {"checkpoint_every": every, "paths": {}}
    runs = (("fp32", "fp32", 0, 0.0), ("bf16_refine", "bf16", w.refine_iters, 0.0),
            ("bf16_triggered", "bf16", w.refine_iters, 0.02))
    traces = {}
    for name, prec, refine, tol in runs:
        st = Alg1Step(w, X, F0d, G0d, B0d, prec, refine, exact_every=every, refine_tol=tol)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(torch.cuda.current_stream())
        tr = st().cpu().numpy()
        e1.record(torch.cuda.current_stream())
        e1.synchronize()
        ck = tr[every - 1::every]
        traces[name] = ck
        rec = {"ms_step_with_checkpoints": round(e0.elapsed_time(e1), 2),
               "checkpoints": [round(float(v), 8) for v in ck],
               "final_tucker_rel_err": float(tr[-1])}
        if prec == "bf16":
            rec["refine_from_sweep"] = st.out.get("refine_from")
            if tol:
                rec["refine_tol"] = tol
        out["paths"][name] = rec
    fp32_final = out["paths"]["fp32"]["final_tucker_rel_err"]
    targets = [round(fp32_final * f, 8) for f in (1.10, 1.02, 1.005)]
    v32 = result.get("fp32_comparison", {}).get("value")
    out["targets"] = {}
    for tgt in targets:
        rec = {}
        for name in ("fp32", "bf16_refine"):
            k = sweeps_to_target(traces[name], tgt)
            sweeps = k * every if k else None
            per = (1.0 / v32) if name == "fp32" and v32 else 1.0 / value_bf16
            rec[name] = {"sweeps": sweeps,
                         "seconds_at_timed_rate": round(sweeps * per, 4) if sweeps else None}
        out["targets"][str(tgt)] = rec
    k = sweeps_to_target(traces["fp32"], out["paths"]["bf16_refine"]["final_tucker_rel_err"])
    out["fp32_sweeps_to_bf16_final_error"] = k * every if k else None
    out["note"] = ("targets are 1.10, 1.02 and 1.005 x the FP32 path's final error; seconds use "
                   "each path's sweeps/s of the timed steps (the BF16 rate includes its refinement "
                   "sweeps); fp32_sweeps_to_bf16_final_error is the first FP32 checkpoint at or "
                   "below the BF16 path's final error")
    return out


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------

def oracle_sample(X64, F0, G0, sweeps):
    """Time `sweeps` oracle nnTD sweeps on the full X; returns (seconds, sweeps)."""
    import oracle
    t0 = time.perf_counter()
    oracle.ntd_fit(X64, F0, G0, sweeps)
    return time.perf_counter() - t0


def line_40cube(dev, steps=5):
    """The 40^3 FP64 workload (planted rank 3, m = 5, 200 + 200 sweeps): the
    whole Alg. 1 step on the FP64 SIMT path (latency-bound: no roofline)."""
    import torch

    from paper_1909_07570_gb300 import inputs
    w = inputs.WORKLOADS["cp3_40x40x40_m5_fp64"]
    X64, _, F0, G0, B0 = inputs.make_problem(w)
    X = torch.tensor(X64, dtype=torch.float64, device=dev)
    F0d = [torch.tensor(f, dtype=torch.float64, device=dev) for f in F0]
    G0d = torch.tensor(G0, dtype=torch.float64, device=dev)
    B0d = [torch.tensor(b, dtype=torch.float64, device=dev) for b in B0]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    step = Alg1Step(w, X, F0d, G0d, B0d, "fp64", 0)
    for _ in range(2):
        step()
    ms = timed_steps(step, steps, flush, torch.cuda.current_stream())
    return {"workload": w.name, "dims": list(w.dims), "m": list(w.m), "r": w.r,
            "ntd_sweeps_per_step": w.iters, "nncp_sweeps_per_step": w.cp_iters, "steps": steps,
            "value": round(w.iters * steps / (sum(ms) / 1e3), 3), "unit": "iters/s",
            "ms_per_step": round(sum(ms) / steps, 4),
            "final_tucker_rel_err": step.tucker_rel_err(),
            "final_lifted_rel_err": step.out["lifted_rel_err"]}


def line_256cube(dev, steps=5):
    """The 256^3 FP32 workload (rank 10, m = 20, 500 + 500 sweeps): the whole
    Alg. 1 step on the TF32x3 passes, device time, and its pass rooflines."""
    import torch

    from paper_1909_07570_gb300 import inputs, native
    w = inputs.WORKLOADS["cp10_256x256x256_m20_fp32"]
    X64, _, F0, G0, B0 = inputs.make_problem(w)
    X = torch.tensor(X64, dtype=torch.float32, device=dev)
    del X64
    F0d = [torch.tensor(f, dtype=torch.float32, device=dev) for f in F0]
    G0d = torch.tensor(G0, dtype=torch.float32, device=dev)
    B0d = [torch.tensor(b, dtype=torch.float32, device=dev) for b in B0]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    step = Alg1Step(w, X, F0d, G0d, B0d, "fp32", 0)
    for _ in range(2):
        step()
    ms = timed_steps(step, steps, flush, torch.cuda.current_stream())
    native.nnc_profile_enable(True)
    step()
    torch.cuda.synchronize()
    prof = {k: native.nnc_profile_read(k) for k in native.PASS_KINDS}
    native.nnc_profile_enable(False)
    peaks, src = load_peaks()
    return {"workload": w.name, "dims": list(w.dims), "m": list(w.m), "r": w.r,
            "ntd_sweeps_per_step": w.iters, "steps": steps,
            "value": round(w.iters * steps / (sum(ms) / 1e3), 3), "unit": "iters/s",
            "ms_per_step": round(sum(ms) / steps, 4),
            "final_tucker_rel_err": step.tucker_rel_err(),
            "final_lifted_rel_err": step.out["lifted_rel_err"],
            "pass_rooflines": pass_rooflines(prof, w, 4, peaks, src, w.name)}


def precision_form(dev):
    """BF16 + FP32-refinement vs FP32 (TF32x3) nnTD on the 512^3 precision
    workload: sweeps/s of device time and the final relative error of each."""
    import torch

    from paper_1909_07570_gb300 import inputs, native
    w = inputs.WORKLOADS["cp16_512x512x512_m32_bf16"]
    X64, _, F0, G0, _ = inputs.make_problem(w)
    X = torch.tensor(X64, dtype=torch.float32, device=dev)
    del X64
    out = {"workload": w.name, "dims": list(w.dims), "m": list(w.m), "sweeps": w.iters,
           "refine_sweeps": w.refine_iters}
    stream = torch.cuda.current_stream()
    for name, prec, refine in (("bf16_refine", "bf16", w.refine_iters), ("fp32", "fp32", 0),
                               ("fp32_simt", "fp32_simt", 0)):
        best, err = None, None
        for _ in range(2):
            F = [torch.tensor(f, dtype=torch.float32, device=dev) for f in F0]
            G = torch.tensor(G0, dtype=torch.float32, device=dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            err, _ = native.ntd_fit(X, F, G, w.iters, precision=prec, refine_iters=refine,
                                    trace=True, rel_err=True)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        out[name] = {"iters_per_s": round(w.iters / (best / 1e3), 2), "ms": round(best, 2),
                     "final_rel_err": err}
    out["bf16_speedup_vs_fp32"] = round(out["bf16_refine"]["iters_per_s"] /
                                        out["fp32"]["iters_per_s"], 3)
    out["abs_rel_err_diff_bf16_vs_fp32"] = abs(out["bf16_refine"]["final_rel_err"] -
                                              out["fp32"]["final_rel_err"])
    return out


def differentiation_form(dev):
    """Block projected-gradient steps on the lifted loss (the hand-written
    adjoint, two TF32x3 passes over X per step) on the 4-way 128^3 x 64
    workload: steps/s of device time (marginal over the setup) and the fit."""
    import numpy as np
    import torch

    from paper_1909_07570_gb300 import inputs, native
    w = inputs.WORKLOADS["cp12_128x128x128x64_m24_fp32"]
    X64, _, F0, _, B0 = inputs.make_problem(w)
    X = torch.tensor(X64, dtype=torch.float32, device=dev)
    xn = float(np.sqrt(np.sum(X64 * X64)))
    del X64
    stream = torch.cuda.current_stream()

    def run(steps):
        F = [torch.tensor(f, dtype=torch.float32, device=dev) for f in F0]
        B = [torch.tensor(b, dtype=torch.float32, device=dev) for b in B0]
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        loss, _ = native.candelinc_pg_fit(X, F, B, steps, precision="fp32")
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), loss

    run(2)
    short = min(run(10)[0] for _ in range(2))
    full, loss = min(run(w.iters) for _ in range(2))
    per_step = (full - short) / (w.iters - 10)
    return {"workload": w.name, "dims": list(w.dims), "m": list(w.m), "r": w.r,
            "steps": w.iters, "ms": round(full, 2),
            "steps_per_s": round(1e3 / per_step, 2),
            "x_bytes_per_step": 2 * int(np.prod(w.dims)) * 4,
            "final_lifted_rel_err": float(np.sqrt(2 * max(loss, 0.0)) / xn)}


def ntd_4way(dev):
    """nnTD of the 4-way 128^3 x 64 workload (two TF32x3 passes over X per
    sweep, the d-way mode-product sweep): sweeps/s of device time (marginal
    over the setup) and the final relative error."""
    import numpy as np
    import torch

    from paper_1909_07570_gb300 import inputs, native
    w = inputs.WORKLOADS["cp12_128x128x128x64_m24_fp32"]
    X64, _, F0, G0, _ = inputs.make_problem(w)
    X = torch.tensor(X64, dtype=torch.float32, device=dev)
    del X64
    stream = torch.cuda.current_stream()

    def run(sweeps):
        F = [torch.tensor(f, dtype=torch.float32, device=dev) for f in F0]
        G = torch.tensor(G0, dtype=torch.float32, device=dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, tr = native.ntd_fit(X, F, G, sweeps, precision="fp32", rel_err=False)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), float(tr[-1])

    run(2)
    short = min(run(10)[0] for _ in range(2))
    full, err = min(run(w.iters) for _ in range(2))
    per_sweep = (full - short) / (w.iters - 10)
    return {"workload": w.name, "dims": list(w.dims), "m": list(w.m), "sweeps": w.iters,
            "ms": round(full, 2), "sweeps_per_s": round(1e3 / per_sweep, 2),
            "x_bytes_per_sweep": 2 * int(np.prod(w.dims)) * 4, "final_rel_err": err}


def batching_form(dev):
    """Many uneven nnTD problems (the batching workload: 64 planted tensors with
    modes in [32, 256], m = 2r) through ntd_fit_batched, then every core fitted
    at CP ranks 2..8 with 8 restarts in one nncp_core_fit_batched launch. Wall
    time around the calls (both return after their work is done)."""
    import torch

    from paper_1909_07570_gb300 import inputs, native
    B = inputs.BATCH
    probs = inputs.batch_problems()

    def upload():
        return [(torch.tensor(p["X"], dtype=torch.float32, device=dev),
                 [torch.tensor(f, dtype=torch.float32, device=dev) for f in p["F0"]],
                 torch.tensor(p["G0"], dtype=torch.float32, device=dev)) for p in probs]

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, out

    warm = upload()[:4]
    native.ntd_fit_batched(warm, 5, precision="fp32", trace=False)
    batch = upload()
    t_ntd, (errs, _, _) = timed(lambda: native.ntd_fit_batched(
        batch, B["iters"], precision="fp32", concurrency=8, trace=False))
    seq = upload()[:8]
    t_seq, _ = timed(lambda: native.ntd_fit_batched(seq, B["iters"], precision="fp32",
                                                     concurrency=1, trace=False))
    def core_jobs():
        jobs = []
        for b, (_, _, G) in enumerate(batch):
            for _, _, B0 in inputs.batch_core_inits(probs[b]["m"], b):
                jobs.append((G, [torch.tensor(x, dtype=torch.float32, device=dev) for x in B0]))
        return jobs

    # The core fits with the launch-shape autotuner off (256 threads per job)
    # and on (its first call tries 32 .. 256 threads on the fit's first sweeps).
    was = native.nnc_autotune_enable(False)
    jobs = core_jobs()
    t_cp256, _ = timed(lambda: native.nncp_core_fit_batched(jobs, B["cp_iters"],
                                                            precision="fp32"))
    native.nnc_autotune_enable(True)
    jobs = core_jobs()
    t_cp, cp_errs = timed(lambda: native.nncp_core_fit_batched(jobs, B["cp_iters"],
                                                               precision="fp32"))
    native.nnc_autotune_enable(was)
    n = len(batch)
    return {"workload": B["name"], "tensors": n, "ntd_sweeps": B["iters"], "concurrency": 8,
            "ntd_ms": round(t_ntd * 1e3, 1), "tensors_per_s": round(n / t_ntd, 2),
            "ntd_sweeps_per_s": round(n * B["iters"] / t_ntd, 1),
            "sequential_first8_ms": round(t_seq * 1e3, 1),
            "batched_speedup_vs_sequential": round((t_seq / 8) / (t_ntd / n), 2),
            "core_fits": len(jobs), "cp_iters": B["cp_iters"],
            "core_fits_ms": round(t_cp * 1e3, 1), "core_fits_per_s": round(len(jobs) / t_cp, 1),
            "core_fits_ms_untuned_256_threads": round(t_cp256 * 1e3, 1),
            "mean_tucker_rel_err": round(float(sum(errs) / n), 6),
            "mean_core_fit_rel_err": round(float(cp_errs.mean().item()), 6)}


def multirank_study(dev, starts=1000, iters=5000):
    """The multirank study of Sec. 4.3 on Ex. "equal": Alg. 1 and Alg. 2 from
    `starts` random starts at multiranks [3,3,3], [3,4,4], [4,4,4], [5,5,5],
    `iters` sweeps per stage (the paper's 5000), all starts of a stage in one
    launch. Reports wall time and the distribution summaries."""
    import torch

    from paper_1909_07570_gb300 import study
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = study.run(starts=starts, iters=iters, device=str(dev))
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    fits = 2 * len(res) // 2 * starts
    return {"tensor": "Ex. equal (4x4x4, rank 4)", "starts": starts, "iters": iters,
            "seconds": round(t, 2), "decompositions_per_s": round(fits / t, 1),
            "summary": study.summary(res)}


def paper_batch(dev):
    """The batch experiment of Sec. 4.3 at the paper's size (1000 planted 40^3
    tensors, canonical multirank (3, 4, 5), rank 5, 5000 sweeps per stage,
    both algorithms) in FP32: device time of each batched stage (CUDA events),
    decompositions per second, and the score summary."""
    import torch

    from paper_1909_07570_gb300 import inputs, study
    probs = inputs.paper_batch_problems()
    study.run_paper_batch(probs[:4], iters=10, dtype=torch.float32, device=dev)
    t = {}
    res = study.run_paper_batch(probs, dtype=torch.float32, device=dev, timings=t)
    gpu_ms = sum(t.values())
    pb = inputs.PAPER_BATCH
    return {"workload": pb["name"], "tensors": len(probs), "sweeps_per_stage": pb["iters"],
            "stage_ms": {k: round(v, 2) for k, v in t.items()}, "gpu_s": round(gpu_ms / 1e3, 3),
            "decompositions_per_s": round(2 * len(probs) / (gpu_ms / 1e3), 1),
            "summary": study.summary_batch(res)}


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(X64, F0, G0, budget_s=20.0):
    secs = oracle_sample(X64, F0, G0, 1)
    n = max(1, min(20, int(budget_s / max(secs, 1e-3)) - 1))
    secs_n = oracle_sample(X64, F0, G0, n)
    return {"value": round(n / secs_n, 4), "unit": "iters/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": f"{n} FP64 oracle nnTD sweeps (numpy) on the full workload tensor; "
                      f"nnCP/lift/residual not included"}


def run_reference(args, rank, world):
    from paper_1909_07570_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    X64, _, F0, G0, _ = inputs.make_problem(w)
    secs = oracle_sample(X64, F0, G0, 1)
    # Each step a bounded sample: about 2 minutes of oracle work in all.
    budget = min(20.0, 120.0 / max(1, args.steps + args.warmup))
    sweeps = max(1, min(10, int(budget / max(secs, 1e-3))))
    for _ in range(args.warmup):
        oracle_sample(X64, F0, G0, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_sample(X64, F0, G0, sweeps)
    total = time.perf_counter() - t0
    value = args.steps * sweeps / total
    sample = f"{sweeps} FP64 oracle nnTD sweeps per step on the full workload tensor"
    return {
        "metric": METRIC, "value": round(value, 4), "unit": "iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded planted nonnegative CP + uniform noise)",
        "config": {"workload": args.workload, "dims": list(w.dims), "m": list(w.m), "r": w.r},
        "impl": "reference",
        "cpu_baseline": {"value": round(value, 4), "unit": "iters/s", "cores": cpu_cores(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "iters/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    rank, world = dist_init(args)
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args, rank, 1)))
        return 0
    result, problem = run_native(args, rank, world)
    if rank == 0 and world == 1 and not args.no_256cube:
        import torch
        result["fp32_256cube"] = line_256cube(torch.device("cuda", 0))
        result["fp64_40cube"] = line_40cube(torch.device("cuda", 0))
    if rank == 0 and world == 1 and not args.no_precision_form:
        import torch
        result["precision_form"] = precision_form(torch.device("cuda", 0))
    if rank == 0 and world == 1 and not args.no_differentiation_form:
        import torch
        result["differentiation_form"] = differentiation_form(torch.device("cuda", 0))
    if rank == 0 and world == 1 and not args.no_4way_ntd:
        import torch
        result["ntd_4way"] = ntd_4way(torch.device("cuda", 0))
    if rank == 0 and world == 1 and not args.no_batching_form:
        import torch
        result["batching_form"] = batching_form(torch.device("cuda", 0))
    if rank == 0 and world == 1 and not args.no_paper_batch:
        import torch
        result["paper_batch"] = paper_batch(torch.device("cuda", 0))
    if rank == 0 and world == 1 and not args.no_multirank_study:
        import torch
        result["multirank_study"] = multirank_study(torch.device("cuda", 0))
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            X64, F0, G0, _ = problem
            result["cpu_baseline"] = cpu_baseline(X64, F0, G0)
        print(json.dumps(result))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
