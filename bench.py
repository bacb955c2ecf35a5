"""Benchmark: all-mode CP gradient + fast CP_ALS on the 4-D 100^4, R = 10 FP32 workload.

One step = one all-mode gradient (Algorithm 2) at the starting factors plus
50 fast CP_ALS sweeps (Section 4) from that start, on a seeded rank-10 CP
model with N(0,1) factors plus 20 dB Gaussian noise (400 MB tensor, larger
than L2, so no flush is needed between steps).

value = algorithmic GFLOP/s of the step (2 flops per multiply-add of the
method's contractions; the R x R solves are not counted), timed with CUDA
events on the launch stream between barriers.  e2e = the same metric with
the tensor copied host->device and the results copied back inside every step.
The roofline object reports the leading contraction (the kernel that streams
Y, about 99% of the step's bytes): algorithmic bytes per launch = 4 * prod(I)
over the event-timed duration of each of its launches, taken in a second run
of the same K steps right after the timed one (events between kernels end the
launch overlap of consecutive kernels, so they stay out of the step timing).

--impl reference times the FP64 CPU oracle (explicit unfoldings and
Khatri-Rao products, Algorithm 1 + eq. 2.14) on the same workload, a bounded
sample per step (one all-mode gradient and one ALS sweep).

After the headline, "configs" measures every workload of the list (3-D FP64
30x40x50, 100^4 R=10, 15^7 R=10/20 with collinear factors, 60^5 R=32/64,
and the 256-member batch) at every precision that applies: gradient and
CP_ALS sweep times, the leading passes' GB/s and roofline fractions, the
error against the FP64 oracle, and the SM clocks seen (--no-configs skips it).
"""
from __future__ import annotations

import argparse
import ctypes
import glob
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import cpsynth  # noqa: E402

WORKLOAD = "cp4d_100_r10_fp32"
ALS_ITERS = 50
METRIC = "all-mode CP-gradient GFLOP/s, % roofline; CP-ALS iter/s at stated rel. error"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def prod(v):
    p = 1
    for x in v:
        p *= int(x)
    return p


def split_point(I):
    best = 0
    for n in range(1, len(I) + 1):
        if prod(I[:n]) <= prod(I[n:]):
            best = n
    return min(max(best, 1), len(I) - 1)


def gradient_flops(I, R):
    """2 flops per multiply-add of Algorithm 2: both leading contractions over
    all of Y, then each recursion and finishing contraction over R^(n)/L^(n)."""
    N, k, P = len(I), split_point(I), prod(I)
    f = 2 * 2 * R * P
    for n in range(k, 0, -1):          # right side: R^(n) has prod(I[:n]) entries per rank
        f += 2 * R * prod(I[:n]) * (2 if n > 1 else 1)
    for n in range(k, N):              # left side: L^(n) has prod(I[n:]) entries per rank
        f += 2 * R * prod(I[n:]) * (2 if n < N - 1 else 1)
    return f


def als_sweep_flops(I, R):
    """One fast ALS sweep: the two leading passes plus the chain contractions."""
    return gradient_flops(I, R)


def step_flops(I, R, iters):
    return gradient_flops(I, R) + iters * als_sweep_flops(I, R)


# ---- ranks (replicas: each rank decomposes its own tensor, no data-path collective) ----
def rank_seed(rank):
    """Seed of the tensor that rank `rank` decomposes (independent problems)."""
    return cpsynth.DEFAULT_SEED + int(rank)


def max_over_ranks(values, device=None):
    """Element-wise maximum of `values` over all ranks of the initialised
    process group (the job takes as long as its slowest rank); the values
    themselves when there is no group or a single rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_value(flops_per_rank_step, world, ms):
    """Whole-job GFLOP/s: every rank's step flops over the slowest rank's step time."""
    return world * flops_per_rank_step / (ms / 1e3) / 1e9


# ---- clocks ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"cpgrad_clocks_gpu{index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- CPU oracle baseline ------------------------------------------------------------------
def openblas_threads():
    """Threads numpy's BLAS will use (its OpenBLAS build), else the CPU count."""
    try:
        import numpy.linalg  # noqa: F401
        libs = [ln.split()[-1] for ln in open("/proc/self/maps") if "openblas" in ln.lower()]
        for path in dict.fromkeys(libs):
            L = ctypes.CDLL(path)
            for sym in ("scipy_openblas_get_num_threads64_", "openblas_get_num_threads64_",
                        "openblas_get_num_threads", "scipy_openblas_get_num_threads"):
                if hasattr(L, sym):
                    fn = getattr(L, sym)
                    fn.restype = ctypes.c_int
                    return int(fn())
    except Exception:
        pass
    return os.cpu_count() or 1


def oracle_sample(p):
    """One all-mode gradient (Algorithm 1 per mode) + one ALS sweep of the oracle; seconds."""
    import oracle
    y = p.y.astype(np.float64)
    t0 = time.perf_counter()
    oracle.cp_gradient_all(y, p.I, p.init)
    oracle.cp_als(y, p.I, p.init, iters=1)
    return time.perf_counter() - t0


def cpu_baseline(p, budget_s=10.0):
    """The oracle's gradient + sweep sample, repeated until about `budget_s`
    seconds of CPU work have run (at least once); mean time per sample."""
    times = []
    while not times or sum(times) < budget_s:
        times.append(oracle_sample(p))
    dt = sum(times) / len(times)
    flops = gradient_flops(p.I, p.R) + als_sweep_flops(p.I, p.R)
    return {"value": flops / dt / 1e9, "unit": "GFLOP/s", "cores": openblas_threads(), "nproc": os.cpu_count(),
            "kind": "oracle",
            "sample": f"{len(times)} x (one all-mode gradient + one ALS sweep) of the FP64 oracle on the full "
                      f"{p.I} R={p.R} tensor, {sum(times):.1f} s in all, {dt:.2f} s each; flops counted as for "
                      f"the GPU step"}


# ---- reference arm -----------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    p = cpsynth.workload(WORKLOAD)
    for _ in range(args.warmup):
        oracle_sample(p)
    times = [oracle_sample(p) for _ in range(args.steps)]
    flops = gradient_flops(p.I, p.R) + als_sweep_flops(p.I, p.R)
    ms = 1e3 * sum(times) / len(times)
    v = flops / (ms / 1e3) / 1e9
    cores = openblas_threads()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "4-D FP32 tensor 100x100x100x100 (rank-10 CP model + 20 dB noise), R=10, "
                                   "oracle step = one all-mode gradient + one ALS sweep", "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": v, "unit": "GFLOP/s", "cores": cores, "nproc": os.cpu_count(), "kind": "oracle",
                             "sample": "each step: one all-mode gradient (Algorithm 1 per mode) + one ALS sweep, "
                                       "full tensor"},
            "e2e": {"value": v, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---- GPU arm ---------------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "tf32x3", "bf16x3", "bf16x6", "bf16"],
                    help="arithmetic of the leading contraction (Algorithm 2 steps 4/7)")
    ap.add_argument("--profile", action="store_true",
                    help="profiling run for ncu: warm-up and timed steps only, no e2e, checks or CPU baseline")
    ap.add_argument("--workload", default="cp4d", choices=["cp4d", "batched"],
                    help="cp4d: the 4-D 100^4 R=10 step (default); batched: many independent tensors per call")
    ap.add_argument("--batch-count", type=int, default=256, help="members of the batched workload")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the per-config measurements (every workload and precision) after the headline")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    import paper_1204_1586_gb300 as cg
    cg.lib()

    # Each rank decomposes its own tensor (independent problems: weak scaling, no data-path collective).
    p = cpsynth.workload(WORKLOAD, seed=rank_seed(rank))
    I, R = p.I, p.R
    Y = torch.from_numpy(p.y).to(dev)
    A0 = [cg.colmajor(torch.from_numpy(a.astype(np.float32)).to(dev)) for a in p.init]
    A = [a.clone() for a in A0]
    G = [torch.empty((R, In), dtype=torch.float32, device=dev).t() for In in I]
    lam = torch.ones(R, dtype=torch.float64, device=dev)
    fit = torch.zeros(ALS_ITERS, dtype=torch.float64, device=dev)
    ws = cg.Workspace(dev)
    stream = torch.cuda.current_stream()

    prec = args.precision

    def step(Yd, A0d=None):
        A0d = A0 if A0d is None else A0d
        cg.cp_gradient_all(Yd, I, A0d, G, workspace=ws, precision=prec)
        for a, a0 in zip(A, A0d):
            a.copy_(a0)
        cg.cp_als_iter(Yd, I, A, ALS_ITERS, lam, fit, workspace=ws, precision=prec)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # The gradient's plan (split k, fused or two passes) is measured once on
    # this data before the warm-up, outside the timed region.
    plan = cg.cp_gradient_autotune(Y, I, A0, G, precision=prec, workspace=ws, reps=3)
    # So is the CP_ALS sweep's split (A0 keeps its values).
    als_plan = cg.cp_als_autotune(Y, I, A0, precision=prec, workspace=ws, reps=3) \
        if prec not in GRAD_ONLY_PRECS else None
    for _ in range(args.warmup):
        step(Y)
    barrier()

    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    cg.launch_count(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed steps' launches
    e0.record(stream)
    for _ in range(args.steps):
        step(Y)
    e1.record(stream)
    barrier()
    torch.cuda.nvtx.range_pop()
    ms = e0.elapsed_time(e1) / args.steps
    launches = cg.launch_count()
    # The same K steps once more with every leading pass bracketed by CUDA
    # events on its stream: the roofline's kernel durations.  An event between
    # two kernels ends their launch overlap, so this region is not the step time.
    cg.profile_lead(True)
    barrier()
    for _ in range(args.steps):
        step(Y)
    barrier()
    lead = cg.profile_read()
    cg.profile_lead(False)
    clocks = clk.stop()

    if args.profile:
        if rank == 0:
            print(json.dumps({"profile_run": True, "ms_per_step": ms, "gpu_launches": launches}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return 0

    # End to end: every step's tensor and starting factors come from pinned
    # host memory and its factors and fits go back to it, all inside the
    # timed region.  Two device buffers: step i + 1's host->device copy runs
    # on a copy stream while step i computes (the first copy is not hidden).
    Yh = torch.from_numpy(p.y).pin_memory()
    Ad_h = [a.cpu().pin_memory() for a in A0]
    out_h = [torch.empty((R, In), dtype=torch.float32).pin_memory() for In in I]
    fit_h = torch.empty(ALS_ITERS, dtype=torch.float64).pin_memory()
    Ybuf = [torch.empty_like(Y) for _ in range(2)]
    Abuf = [[torch.empty_like(a) for a in A0] for _ in range(2)]
    cstream = torch.cuda.Stream(device=dev)
    ready = [torch.cuda.Event() for _ in range(2)]  # buffer b holds its step's inputs
    free = [torch.cuda.Event() for _ in range(2)]   # the step that used buffer b is done

    def copy_in(b, after=None):
        if after is not None:
            cstream.wait_event(after)
        cstream.wait_event(free[b])
        with torch.cuda.stream(cstream):
            Ybuf[b].copy_(Yh, non_blocking=True)
            for a, h in zip(Abuf[b], Ad_h):
                a.copy_(h, non_blocking=True)
        ready[b].record(cstream)

    def compute(b):
        stream.wait_event(ready[b])
        step(Ybuf[b], Abuf[b])
        for g, h in zip(A, out_h):
            h.copy_(g.t(), non_blocking=True)
        fit_h.copy_(fit, non_blocking=True)
        free[b].record(stream)

    def run_e2e(nsteps, start_event=None):
        copy_in(0, start_event)
        for i in range(nsteps):
            if i + 1 < nsteps:
                copy_in((i + 1) % 2)
            compute(i % 2)

    run_e2e(1)
    barrier()
    e0.record(stream)
    run_e2e(args.steps, e0)
    e1.record(stream)
    barrier()
    ms_e2e = e0.elapsed_time(e1) / args.steps
    h2d = Yh.numel() * 4 + sum(a.numel() * 4 for a in Ad_h)
    d2h = sum(h.numel() * 4 for h in out_h) + fit_h.numel() * 8

    ms, ms_e2e = max_over_ranks([ms, ms_e2e], device=dev)

    flops = step_flops(I, R, ALS_ITERS)
    value = job_value(flops, world, ms)
    value_e2e = job_value(flops, world, ms_e2e)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    hbm, peak_kind = peaks()
    ybytes = 4 * prod(I)
    lead = [(t, s) for t, s in lead if s in (1, 2, 3)]
    lead_ms = [t for t, _ in lead]
    per_side = {}
    for t, s in lead:
        per_side.setdefault({1: "step4_R", 2: "step7_L", 3: "step4+7_fused"}[s], []).append(t)
    avg = sum(lead_ms) / len(lead_ms) if lead_ms else float("nan")
    achieved = ybytes / (avg / 1e3) / 1e9
    # The split forms run the tensor-core kernels (J = 10^4 rows are whole 16-byte chunks).
    kernel = {"fp32": "lead_simt_kernel", "tf32x3": "lead_tf32_kernel"}.get(prec, "lead_ws_kernel")
    traffic = lead_traffic(kernel)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "peak_kind": peak_kind, "kernel": f"{kernel} (Algorithm 2 steps 4/7)",
                "launches": len(lead_ms),
                "per_variant_GBps": {k: ybytes / (sum(v) / len(v) / 1e3) / 1e9 for k, v in per_side.items()}}

    check = {}
    if not args.no_check:
        import oracle
        Gc = cg.cp_gradient_all(Y, I, A0, workspace=ws, precision=prec)
        torch.cuda.synchronize()
        want = oracle.cp_gradient_all(p.y.astype(np.float64), I, p.init)
        check["gradient_rel_err_max"] = max(
            float(np.linalg.norm(Gc[n].double().cpu().numpy() - want[n]) / np.linalg.norm(want[n]))
            for n in range(len(I)))
        Ac = [a.clone() for a in A0]
        _, fc = cg.cp_als_iter(Y, I, Ac, 2, workspace=ws, precision=prec)
        tr = oracle.cp_als(p.y.astype(np.float64), I, p.init, iters=2)
        check["als_fit_abs_err_2sweeps"] = float(np.max(np.abs(fc.cpu().numpy() - np.array(tr.fits))))
        check["als_final_fit"] = float(fit.cpu().numpy()[-1])

    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "4-D FP32 tensor 100x100x100x100, rank-10 CP model (N(0,1) factors) + 20 dB noise, "
                               "R=10: one all-mode gradient + 50 fast CP_ALS sweeps per step",
                   "I": I, "R": R, "split_k": split_point(I), "precision": prec, "als_iters": ALS_ITERS,
                   "gradient_plan": {"split": plan["split"], "fused": plan["fused"], "tuned_ms": plan["ms"],
                                     "candidates": plan["candidates"]},
                   "als_plan": None if als_plan is None else {"split": als_plan["split"], "tuned_ms": als_plan["ms"],
                                                              "candidates": als_plan["candidates"]},
                   "l2": "inputs larger than L2 (400 MB tensor)", "parallelism": "replicas" if world > 1 else "1 GPU"},
        "gradient_gflops": gradient_flops(I, R) / 1e9,
        "als_iter_per_s": None,
        "roofline": roofline,
        "e2e": {"value": value_e2e, "unit": "GFLOP/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "note": "each step's inputs copied from pinned host memory inside the timed region, double-buffered: "
                        "step i+1's copy overlaps step i's compute"},
        "gpu_launches": launches,
        "clocks": clocks,
        "check": check,
    }
    # Every launch of one more step, event-timed one by one on its stream
    # (outside the timed region): where a step's time goes, per kind of kernel.
    cg.profile_lead(2)
    step(Y)
    torch.cuda.synchronize()
    rec = cg.profile_read()
    cg.profile_lead(False)
    brk = {}
    for t, kind in rec:
        name = cg.LAUNCH_KINDS.get(kind, str(kind))
        e = brk.setdefault(name, {"launches": 0, "us": 0.0})
        e["launches"] += 1
        e["us"] += 1e3 * t
    line["step_breakdown"] = {"note": "one step, each launch bracketed by CUDA events (kernel time; the rest "
                                      "of the step is launch gaps)", "kinds": brk,
                              "kernel_us_total": sum(e["us"] for e in brk.values())}
    # per-component timing outside the timed region (informational)
    tg = _time_component(lambda: cg.cp_gradient_all(Y, I, A0, G, workspace=ws, precision=prec), stream)
    ta = _time_component(lambda: cg.cp_als_iter(Y, I, [a.clone() for a in A0], 10, workspace=ws, precision=prec),
                         stream) / 10
    line["gradient_ms"] = tg
    line["gradient_gflops"] = gradient_flops(I, R) / (tg / 1e3) / 1e9
    line["gradient_frac_of_one_pass_roofline"] = (ybytes / hbm / 1e6) / tg
    line["als_iter_per_s"] = 1e3 / ta
    line["als_frac_of_two_pass_roofline"] = (2 * ybytes / hbm / 1e6) / ta
    # The gradient's consumers on the same tensor (informational): the cost
    # gradient of eq. 2.13, one first-order step (eq. 2.15), and multiplicative
    # NTF sweeps (eq. 2.18) on |Y| with nonnegative factors.
    line["cost_gradient_ms"] = _time_component(
        lambda: cg.cp_gradient_full(Y, I, A0, G, workspace=ws, precision=prec), stream)
    Ast = [a.clone() for a in A0]
    line["gradient_step_ms"] = _time_component(
        lambda: cg.cp_gradient_step(Y, I, Ast, 1e-9, G, workspace=ws, precision=prec), stream)
    Yabs = Y.abs()
    Ann = [cg.colmajor(a.abs()) for a in A0]
    line["ntf_sweep_ms"] = _time_component(
        lambda: cg.cp_ntf_iter(Yabs, I, [a.clone() for a in Ann], 5, workspace=ws, precision=prec), stream) / 5
    del Yabs
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p)
    if not args.no_configs:
        del Ast
        try:
            line["configs"] = measure_configs(cg, dev, stream, hbm, args.batch_count)
        except Exception as ex:  # keep the headline line whatever happens here
            line["configs"] = {"error": f"{type(ex).__name__}: {str(ex)[:300]}"}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


LEAD_KERNELS = {
    # kernel family -> (sources whose hash identifies the captured build, traffic summary)
    "lead_simt_kernel": (("lead_simt.cuh", "common.cuh", "tc_common.cuh"), "lead_simt_traffic.json"),
    "lead_ws_kernel": (("lead_ws.cuh", "tc_common.cuh", "common.cuh"), "lead_ws_traffic.json"),
    "lead_tf32_kernel": (("lead_tf32.cuh", "lead_ws.cuh", "tc_common.cuh", "common.cuh"), "lead_tf32_traffic.json"),
}


# ---- every config of the workload list, every precision (informational keys) -----------
SWEEP_PRECS = ("fp32", "tf32x3", "bf16x6")      # CP_ALS precisions
GRAD_ONLY_PRECS = ("bf16x3", "bf16")            # gradient-only precisions


def _rel_err_max(G, want):
    return max(float(np.linalg.norm(G[n].double().cpu().numpy() - want[n]) / np.linalg.norm(want[n]))
               for n in range(len(want)))


def _measure_case(cg, Y, I, A0, G, ws, stream, prec, hbm, esize=4):
    """Gradient (autotuned plan) and CP_ALS sweep times of one tensor at one
    precision, the leading passes' GB/s (event-timed launch by launch), and
    the fractions of the one-pass (gradient) and two-pass (sweep) floors."""
    ybytes = esize * prod(I)
    out = {}
    plan = cg.cp_gradient_autotune(Y, I, A0, G, precision=prec, workspace=ws, reps=2)
    out["gradient_plan"] = {"split": plan["split"], "fused": plan["fused"]}
    tg = _time_component(lambda: cg.cp_gradient_all(Y, I, A0, G, workspace=ws, precision=prec), stream)
    out["gradient_ms"] = tg
    out["gradient_frac_of_one_pass_roofline"] = (ybytes / hbm / 1e6) / tg
    cg.profile_lead(1)
    cg.cp_gradient_all(Y, I, A0, G, workspace=ws, precision=prec)
    passes = {}
    if prec not in GRAD_ONLY_PRECS:
        ap = cg.cp_als_autotune(Y, I, A0, precision=prec, workspace=ws, reps=2)
        out["als_plan"] = {"split": ap["split"], "candidates": ap["candidates"]}
        ta = _time_component(lambda: cg.cp_als_iter(Y, I, [a.clone() for a in A0], 5, workspace=ws, precision=prec),
                             stream) / 5
        out["als_sweep_ms"] = ta
        out["als_frac_of_two_pass_roofline"] = (2 * ybytes / hbm / 1e6) / ta
        cg.profile_lead(1)
        cg.cp_als_iter(Y, I, [a.clone() for a in A0], 3, workspace=ws, precision=prec)
    import torch
    torch.cuda.synchronize()
    for t, k in cg.profile_read():
        name = {1: "step4_R", 2: "step7_L", 3: "step4+7_fused"}.get(k)
        if name:
            passes.setdefault(name, []).append(t)
    cg.profile_lead(False)
    out["pass_GBps"] = {k: ybytes / (statistics.median(v) / 1e3) / 1e9 for k, v in passes.items()}
    out["pass_frac"] = {k: v / hbm for k, v in out["pass_GBps"].items()}
    return out


def measure_configs(cg, dev, stream, hbm, batch_count):
    """Every config of the workload list (the 3-D FP64 correctness case, 100^4
    R=10, 15^7 R=10/20, 60^5 R=32/64, the 256-member batch), each at every
    precision that applies, with its error against the FP64 oracle (every
    entry, or 100 sampled entries of eq. 3.2 at 60^5) and the SM clocks seen
    while it ran.  Informational: the headline value stays the 100^4 step."""
    import torch
    import oracle
    res = {}
    ws = cg.Workspace(dev)

    def colmaj(a):
        return cg.colmajor(torch.from_numpy(np.asarray(a, dtype=np.float32)).to(dev))

    def run_config(name, fn):
        clk = ClockSampler(dev.index or 0)
        clk.start()
        t0 = time.time()
        try:
            r = fn()
        except Exception as ex:
            r = {"error": f"{type(ex).__name__}: {str(ex)[:200]}"}
        r["clocks"] = clk.stop()
        r["wall_s"] = round(time.time() - t0, 1)
        res[name] = r

    # 3-D FP64 30x40x50, R=5: latency-bound correctness case (times in us)
    def c3d():
        p = cpsynth.workload("cp3d_30x40x50_r5_fp64")
        Y = torch.from_numpy(p.y).to(dev)
        A0 = [cg.colmajor(torch.from_numpy(a).to(dev)) for a in p.init]
        G = [torch.empty((p.R, In), dtype=torch.float64, device=dev).t() for In in p.I]
        cg.cp_gradient_all(Y, p.I, A0, G, workspace=ws, precision="fp64")
        want = oracle.cp_gradient_all(p.y, p.I, p.init)
        err = _rel_err_max(G, want)
        tg = _time_component(lambda: cg.cp_gradient_all(Y, p.I, A0, G, workspace=ws, precision="fp64"), stream)
        A = [a.clone() for a in A0]
        _, fit = cg.cp_als_iter(Y, p.I, A, 10, workspace=ws, precision="fp64")
        tr = oracle.cp_als(p.y, p.I, p.init, iters=10)
        ta = _time_component(lambda: cg.cp_als_iter(Y, p.I, [a.clone() for a in A0], 10, workspace=ws,
                                                    precision="fp64"), stream) / 10
        return {"precision": "fp64", "gradient_us": 1e3 * tg, "als_sweep_us": 1e3 * ta,
                "gradient_rel_err_max": err,
                "als_fit_abs_err_10_sweeps": float(np.max(np.abs(fit.cpu().numpy() - np.array(tr.fits))))}
    run_config("cp3d_30x40x50_r5_fp64", c3d)

    # 100^4 R=10 and 15^7 R=10/20: every precision, every entry against the oracle
    for wname in ("cp4d_100_r10_fp32", "cp7d_15_r10_fp32", "cp7d_15_r20_fp32"):
        def cfull(wname=wname):
            p = cpsynth.workload(wname)
            Y = torch.from_numpy(p.y).to(dev)
            A0 = [colmaj(a) for a in p.init]
            G = [torch.empty((p.R, In), dtype=torch.float32, device=dev).t() for In in p.I]
            want = oracle.cp_gradient_all(p.y, p.I, [a.astype(np.float32).astype(np.float64) for a in p.init])
            out = {}
            for prec in SWEEP_PRECS + GRAD_ONLY_PRECS:
                r = _measure_case(cg, Y, p.I, A0, G, ws, stream, prec, hbm)
                cg.cp_gradient_all(Y, p.I, A0, G, workspace=ws, precision=prec)
                r["gradient_rel_err_max"] = _rel_err_max(G, want)
                out[prec] = r
            return out
        run_config(wname.replace("_fp32", ""), cfull)

    # 60^5 R=32/64: one N(0,1) tensor; errors from 100 sampled entries (eq. 3.2)
    I5 = [60] * 5
    y5 = cpsynth.random_tensor(I5, seed=cpsynth.DEFAULT_SEED + 50)
    Y5 = torch.from_numpy(y5).to(dev)
    for R in (32, 64):
        def c5d(R=R):
            A = cpsynth.random_factors(I5, R, seed=cpsynth.DEFAULT_SEED + R)
            A0 = [colmaj(a) for a in A]
            G = [torch.empty((R, In), dtype=torch.float32, device=dev).t() for In in I5]
            rng = np.random.default_rng(R)
            samples = []
            for n in range(5):
                pairs = sorted((int(rng.integers(60)), int(rng.integers(R))) for _ in range(20))
                samples.append((pairs, oracle.cp_gradient_entries(y5, I5, A, n, pairs)))
            out = {}
            for prec in SWEEP_PRECS + GRAD_ONLY_PRECS:
                r = _measure_case(cg, Y5, I5, A0, G, ws, stream, prec, hbm)
                cg.cp_gradient_all(Y5, I5, A0, G, workspace=ws, precision=prec)
                errs = []
                for n, (pairs, ref) in enumerate(samples):
                    Gn = G[n].double().cpu().numpy()
                    got = np.array([Gn[i, r_] for i, r_ in pairs])
                    errs.append(float(np.sqrt(np.mean((got - ref) ** 2) / np.mean(np.square(ref)))))
                r["gradient_rel_err_sampled"] = max(errs)
                out[prec] = r
            return out
        run_config(f"cp5d_60_r{R}", c5d)
    del Y5, y5
    torch.cuda.empty_cache()

    # the 256-member batch: 30 sweeps per member per call; three ways of running it
    def cbatch():
        shapes = cpsynth.batched_shapes(batch_count)
        gen = torch.Generator(device=dev)
        Ys, members, A0s, As = [], [], [], []
        for b, (I, R) in enumerate(shapes):
            gen.manual_seed(cpsynth.DEFAULT_SEED + 1 + b)
            Ys.append(torch.randn(prod(I), generator=gen, device=dev))
            A0 = [colmaj(a) for a in cpsynth.gaussian_factors(I, R, seed=cpsynth.DEFAULT_SEED + 1 + b, stream=1)]
            A0s.append(A0)
            As.append([a.clone() for a in A0])
        entries = sum(prod(I) for I, _ in shapes)
        lams = [torch.ones(R, dtype=torch.float64, device=dev) for _, R in shapes]
        fits = [torch.zeros(BATCH_ITERS, dtype=torch.float64, device=dev) for _ in shapes]
        members = [(Y, I, A, lam, fit) for Y, (I, _), A, lam, fit in zip(Ys, shapes, As, lams, fits)]

        def reset():
            for A, A0 in zip(As, A0s):
                for a, a0 in zip(A, A0):
                    a.copy_(a0)

        def batched():
            reset()
            cg.cp_als_batched(members, BATCH_ITERS, workspace=ws)

        def serial():
            reset()
            for Y, I, A, lam, fit in members:
                cg.cp_als_iter(Y, I, A, BATCH_ITERS, lam, fit, workspace=ws)
        out = {"members": len(shapes), "entries": entries, "bytes": 4 * entries, "precision": "fp32",
               "als_iters": BATCH_ITERS,
               "data": "N(0,1) tensors drawn on the device (seeded per member), shapes and ranks and ALS starts "
                       "from the seeded workload generator; timing only"}
        out["batched_call_ms_nstar"] = _time_component(batched, stream, reps=2)
        # the CP_ALS split of every member, measured (A and lambda keep their values)
        t0 = time.time()
        off = 0
        for Y, I, A, lam, _ in members:
            off += cg.cp_als_autotune(Y, I, A, lam, workspace=ws, reps=1)["split"] != cg.cpg_split_point(I)
        torch.cuda.synchronize()
        out["als_autotune"] = {"seconds": round(time.time() - t0, 2), "members_not_at_nstar": int(off)}
        out["batched_call_ms"] = _time_component(batched, stream, reps=2)
        out["per_member_calls_ms"] = _time_component(serial, stream, reps=1)

        def batched_x6():
            reset()
            cg.cp_als_batched(members, BATCH_ITERS, workspace=ws, precision="bf16x6")
        for Y, I, A, lam, _ in members:
            cg.cp_als_autotune(Y, I, A, lam, workspace=ws, reps=1, precision="bf16x6")
        out["batched_call_ms_bf16x6"] = _time_component(batched_x6, stream, reps=2)
        batched()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            reset()
            cg.cp_als_batched(members, BATCH_ITERS, workspace=ws)
        out["graph_replay_ms"] = _time_component(g.replay, stream, reps=2)
        sweeps = len(shapes) * BATCH_ITERS
        out["sweeps_per_s"] = sweeps / (out["batched_call_ms"] / 1e3)
        out["two_pass_GBps"] = 2 * 4 * entries * BATCH_ITERS / (out["batched_call_ms"] / 1e3) / 1e9
        out["two_pass_frac"] = out["two_pass_GBps"] / hbm
        out["speedup_vs_per_member_calls"] = out["per_member_calls_ms"] / out["batched_call_ms"]
        out["device_status"] = cg.cpg_device_status(ws)
        del g
        return out
    run_config("batched_256", cbatch)
    return res


# ---- batched workload -------------------------------------------------------------------
BATCH_ITERS = 30


def run_batched(args):
    """Many independent tensors (order 3-5, every I_n in [8, 64], R in [4, 32],
    rank-R N(0,1) CP models + 20 dB noise), 30 fast CP_ALS sweeps on each per
    step.  Three ways of running the same work are timed: one cp_als_batched
    call (members on a stream pool), that call captured once in a CUDA graph
    and replayed, and one cp_als_iter call per member on one stream."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1204_1586_gb300 as cg
    t0 = time.time()
    probs = cpsynth.batched_workload(count=args.batch_count)
    gen_s = time.time() - t0
    entries = sum(prod(p.I) for p in probs)
    Ys = [torch.from_numpy(p.y).to(dev) for p in probs]
    # All factors in one flat buffer, so that a step starts from the same
    # point with one device copy.
    sizes = [[In * p.R for In in p.I] for p in probs]
    flat0 = torch.cat([torch.from_numpy(np.ascontiguousarray(a.T).astype(np.float32)).reshape(-1)
                       for p in probs for a in p.init]).to(dev)
    flat = flat0.clone()
    A, o = [], 0
    for p, sz in zip(probs, sizes):
        fac = []
        for In, n in zip(p.I, sz):
            fac.append(flat[o:o + n].view(p.R, In).t())
            o += n
        A.append(fac)
    lams = [torch.ones(p.R, dtype=torch.float64, device=dev) for p in probs]
    fits = [torch.zeros(BATCH_ITERS, dtype=torch.float64, device=dev) for p in probs]
    members = [(Y, p.I, a, lam, fit) for Y, p, a, lam, fit in zip(Ys, probs, A, lams, fits)]
    ws = cg.Workspace(dev)
    stream = torch.cuda.current_stream()

    prec = args.precision

    def step_batched():
        flat.copy_(flat0)
        cg.cp_als_batched(members, BATCH_ITERS, workspace=ws, precision=prec)

    def step_serial():
        flat.copy_(flat0)
        for Y, I, a, lam, fit in members:
            cg.cp_als_iter(Y, I, a, BATCH_ITERS, lam, fit, workspace=ws, precision=prec)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    clk = ClockSampler(0)
    clk.start()
    ms_batched = timed(step_batched, args.steps, args.warmup)
    clocks = clk.stop()
    ms_serial = timed(step_serial, max(1, args.steps // 2), 1)
    ms_graph, graph_note = None, None
    try:
        step_batched()  # workspace and streams exist before capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            cg.cp_als_batched(members, BATCH_ITERS, workspace=ws, precision=prec)
        ms_graph = timed(lambda: (flat.copy_(flat0), g.replay()), args.steps, 2)
    except Exception as ex:  # report, keep the other numbers
        graph_note = f"capture failed: {str(ex)[:160]}"
    status = cg.cpg_device_status(ws)
    sweeps = len(probs) * BATCH_ITERS
    gbytes = 2 * 4 * entries * BATCH_ITERS / 1e9  # two passes over every member per sweep
    line = {
        "metric": "batched CP-ALS sweeps/s (all members)", "value": sweeps / (ms_batched / 1e3), "unit": "sweeps/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batched, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batched: {len(probs)} FP32 tensors, order 3-5, I_n in [8, 64], R in [4, 32], "
                               f"rank-R N(0,1) CP models + 20 dB noise; {BATCH_ITERS} fast CP_ALS sweeps each per step",
                   "members": len(probs), "entries": entries, "bytes": 4 * entries, "als_iters": BATCH_ITERS,
                   "l2": "inputs larger than L2 (%.1f GB)" % (4 * entries / 1e9), "generation_s": round(gen_s, 1),
                   "precision": prec},
        "effective_GBps": gbytes / (ms_batched / 1e3),
        "per_member_calls_ms": ms_serial, "graph_replay_ms": ms_graph, "graph_note": graph_note,
        "speedup_vs_per_member_calls": ms_serial / ms_batched,
        "device_status": status, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def lead_kernel_hash(kernel):
    """Hash of the kernel family's sources with comments and blank space
    removed: it changes when the code does, not when a comment does."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in LEAD_KERNELS[kernel][0]:
        with open(os.path.join(ROOT, "paper_1204_1586_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def lead_traffic(kernel):
    """DRAM bytes per launch of the leading kernel from the committed ncu
    summary, or None when the kernel source changed since it was captured."""
    tf = os.path.join(ROOT, "profiles", LEAD_KERNELS[kernel][1])
    try:
        with open(tf) as f:
            d = json.load(f)
        if d.get("kernel_source_hash") == lead_kernel_hash(kernel):
            return d.get("bytes_per_launch")
    except Exception:
        pass
    return None


def _time_component(fn, stream, reps=5):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


if __name__ == "__main__":
    sys.exit(main())
