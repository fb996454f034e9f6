#!/usr/bin/env python3
"""Benchmark of the structured-grid solver hot path on one GB300 (or N replicas).

One STEP is one pass of the whole hot path over the 3-D Poisson workload
(256^3 interior nodes, 16.8 M unknowns, FP64, rhs ~ U(-1, 1) from seed 0):
  a1  one stencil SpMV y = A b                     (7-point Laplacian)
  a2  Jacobi, 200 sweeps                           (Laplacian)
  a3  lexicographic Gauss-Seidel, 200 sweeps       (Laplacian)
  a4  CG to 1e-10 relative residual from x0 = 0    (Laplacian)
  a5  BiCGStab to 1e-10 from x0 = 0                (7-point upwind
      convection-diffusion, beta = (1, 0.5, 0.25) scaled to cell Peclet 0.5)
value = algorithmic bytes of the step / step time (GB/s), with the inputs
already resident in HBM; e2e = the same metric through the public API with
the right-hand side copied in from pinned host memory and every solution
copied back out inside the timed region.

The path does not shard (each GPU solves its own system): with --gpus N
every rank runs an independent replica ("replicas only", weak scaling).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (rank 0 only).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solver GB/s & % HBM peak; time-to-1e-10 residual, mixed/batched vs plain FP64"

# Algorithmic bytes per unknown (FP64) -- the minimum traffic of each step of
# the method, counting every vector the algorithm must read and write once.
BYTES = {
    "spmv": 16.0,          # read x, write y
    "jacobi": 24.0,        # per sweep: read x, b; write x'
    "gauss_seidel": 24.0,  # per sweep: read x, b; write x (in place)
    "cg": 64.0,            # per iteration: read r, p_old / write p; read x, p, r / write x, r
    "bicgstab": 136.0,     # per iteration (17 vector passes of 8 B)
}

# FP64 flops per unknown and iteration executed by the kernels (FMA = 2),
# counted from the kernel code for the 7-point operators of the workload:
#   spmv      3 pair adds + 3 FMA + 1 scaling multiply             = 10
#   jacobi    3 pair adds + 3 FMA                                   =  9
#   gs        as jacobi                                             =  9
#   cg        p update FMA, stencil 3 adds + 3 FMA, p.w FMA;
#             x and r FMA, r.r FMA                                  = 19
#   bicgstab  p update 2 FMA, upwind stencil 6 FMA, v.r' FMA;
#             s FMA, stencil 6 FMA, 3 dot FMA; x 2 FMA, r FMA,
#             2 dot FMA                                             = 48
FLOPS = {"spmv": 10.0, "jacobi": 9.0, "gauss_seidel": 9.0, "cg": 19.0, "bicgstab": 48.0}

# DRAM bytes per unknown and iteration measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum) on short launches of the same kernels at 256^3
# (profiles/fp64_and_traffic_poisson3d_256.md: CG and BiCGStab 10 iterations,
# Jacobi 20 sweeps, one launch per capture; the start-up residual pass is
# subtracted).  Traffic grows with unknowns x iterations (each pass streams
# every vector), so a launch of the step moves this figure x N x iterations.
# Re-measure whenever the kernel changes.
TRAFFIC_B_PER_UNIT = {"cg": 74.3, "bicgstab": 135.1, "jacobi": 24.9}
# FP64 pipe: 2 FMA lanes per SM per clock (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on
# peak_sustained = 2 per SM per cycle) x 2 flops x 152 SMs.
FP64_FLOPS_PER_CLK = 2 * 2 * 152


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=256, help="grid side (default 256 -> 256^3)")
    p.add_argument("--sweeps", type=int, default=200)
    p.add_argument("--tol", type=float, default=1e-10)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-roofline", action="store_true", help="skip the roofline repeats (profiling runs)")
    p.add_argument("--timeout-s", type=float, default=2.0, help="bound on device-side waits")
    p.add_argument("--mixed-n", type=int, default=512, help="grid side of the mixed-precision comparison (0: skip)")
    p.add_argument("--adjoint-n", type=int, default=256, help="grid side of the adjoint-gradient timing (0: skip)")
    p.add_argument("--batch-n", type=int, default=512, help="systems in the batched comparison (0: skip)")
    p.add_argument("--no-variants", action="store_true", help="skip the CG-NB / BiCGStab-B1 comparison")
    p.add_argument("--hpcg-nz", type=int, default=6144,
                   help="z extent of the HPCG 128 x 128 x nz timing (the paper's node: 6144; 0: skip)")
    p.add_argument("--batch-vark", action="store_true",
                   help="batched comparison: CG systems on variable-k diffusion (log k ~ N(0, 1))")
    return p.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands on a bounded sample
# ---------------------------------------------------------------------------
def oracle_sample(n: int, b: np.ndarray, all_cores: bool = False):
    """Runs the oracle on a bounded sample of the step; returns (bytes, seconds,
    description, threads).  all_cores: the OpenMP build of the same source
    (element-wise loops on every core this process may use; inner products and
    Gauss-Seidel sweeps sequential; bitwise the same results)."""
    import contextlib

    import oracle
    if all_cores and oracle.have_all_cores():
        with oracle.all_cores() as threads:
            nb, secs, desc = _oracle_sample(n, b)
        return nb, secs, desc + "; OpenMP build, %d threads (GS sequential)" % threads, threads
    with contextlib.nullcontext():
        nb, secs, desc = _oracle_sample(n, b)
    return nb, secs, desc + "; single-threaded C oracle", 1


def _oracle_sample(n: int, b: np.ndarray):
    import oracle
    from paper_2305_05988_gb300 import inputs
    shape = (n, n, n)
    N = n ** 3
    A = oracle.Operator(shape)
    U = oracle.Operator(shape, oracle.UPWIND, inputs.upwind_beta(shape, 0.5))
    work = []
    t0 = time.perf_counter()
    A.spmv(b)
    work.append(("spmv", 1, time.perf_counter() - t0))
    t0 = time.perf_counter()
    oracle.jacobi(A, b, maxit=2)
    work.append(("jacobi", 2, time.perf_counter() - t0))
    t0 = time.perf_counter()
    oracle.gauss_seidel(A, b, maxit=2)
    work.append(("gauss_seidel", 2, time.perf_counter() - t0))
    t0 = time.perf_counter()
    oracle.cg(A, b, maxit=2, tol=0.0)
    work.append(("cg", 2, time.perf_counter() - t0))
    t0 = time.perf_counter()
    oracle.bicgstab(U, b, maxit=1, tol=0.0)
    work.append(("bicgstab", 1, time.perf_counter() - t0))
    nbytes = sum(BYTES[k] * N * c for k, c, _ in work)
    secs = sum(t for _, _, t in work)
    desc = ("%d^3: 1 SpMV, 2 Jacobi sweeps, 2 GS sweeps, 2 CG iterations (incl. setup), "
            "1 BiCGStab iteration (incl. setup)" % n)
    return nbytes, secs, desc


# ---------------------------------------------------------------------------
# reference arm
# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2305_05988_gb300 import inputs
    n = args.n
    b = inputs.rhs_uniform((n, n, n), 0)
    for _ in range(args.warmup):
        oracle_sample(n, b, all_cores=True)
    tot_b, tot_s = 0.0, 0.0
    desc, cores = "", 1
    for _ in range(args.steps):
        nb, s, desc, cores = oracle_sample(n, b, all_cores=True)
        tot_b += nb
        tot_s += s
    value = tot_b / tot_s / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "poisson3d %d^3 FP64 (bounded oracle sample per step)" % n},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def replica_throughput(local_bytes, local_ms, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas ("replicas only": no data
    exchange between ranks): the bytes every rank processed over the slowest
    rank's time.  Returns (GB/s, max ms, total bytes)."""
    if dist is None:
        return local_bytes / (local_ms * 1e-3) / 1e9, local_ms, local_bytes
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    nb = torch.tensor([float(local_bytes)], dtype=torch.float64, device=device)
    dist.all_reduce(nb, op=dist.ReduceOp.SUM)
    ms, total = float(t.item()), float(nb.item())
    return total / (ms * 1e-3) / 1e9, ms, total


def run_ours(args, rank, world, dist):
    import torch

    import paper_2305_05988_gb300 as hs
    from paper_2305_05988_gb300 import inputs
    from paper_2305_05988_gb300 import _lib

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.n
    shape = (n, n, n)
    N = n ** 3
    b_host = inputs.rhs_uniform(shape, 0)
    b = torch.from_numpy(b_host).to(dev)
    A = hs.Operator.laplacian(shape)
    beta = inputs.upwind_beta(shape, 0.5)
    U = hs.Operator.upwind(shape, beta)
    stream = torch.cuda.current_stream(dev)
    maxk = 20000
    tmo = args.timeout_s
    # workspaces are allocated once, outside the timed region
    xs = {k: torch.zeros(N, dtype=torch.float64, device=dev) for k in ("y", "jacobi", "gs", "cg", "bicgstab")}

    def step(bv, record=None, on_done=None):
        """One pass of the hot path; on_done(name) runs after each solver (the
        end-to-end loop uses it to start that solution's copy to the host while
        the next solver computes)."""
        info = {}
        done = on_done or (lambda name: None)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)] if record is not None else None
        if ev:
            ev[0].record(stream)
        A.spmv(bv, out=xs["y"])
        done("y")
        if ev:
            ev[1].record(stream)
        xs["jacobi"].zero_()
        _, info["jacobi"] = hs.jacobi(A, bv, xs["jacobi"], maxit=args.sweeps, inplace=True, timeout_s=tmo)
        done("jacobi")
        if ev:
            ev[2].record(stream)
        xs["gs"].zero_()
        _, info["gauss_seidel"] = hs.gauss_seidel(A, bv, xs["gs"], maxit=args.sweeps, inplace=True,
                                                  timeout_s=tmo)
        done("gs")
        if ev:
            ev[3].record(stream)
        xs["cg"].zero_()
        _, info["cg"] = hs.cg(A, bv, xs["cg"], tol=args.tol, maxit=maxk, inplace=True, timeout_s=tmo)
        done("cg")
        if ev:
            ev[4].record(stream)
        xs["bicgstab"].zero_()
        _, info["bicgstab"] = hs.bicgstab(U, bv, xs["bicgstab"], tol=args.tol, maxit=maxk, inplace=True,
                                          timeout_s=tmo)
        done("bicgstab")
        if ev:
            ev[5].record(stream)
            record.append(ev)
        return info

    def step_bytes(info):
        tot = BYTES["spmv"] * N
        tot += BYTES["jacobi"] * N * info["jacobi"].iters
        tot += BYTES["gauss_seidel"] * N * info["gauss_seidel"].iters
        tot += BYTES["cg"] * N * info["cg"].iters
        tot += BYTES["bicgstab"] * N * info["bicgstab"].iters
        return tot

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(max(args.warmup, 0)):
        info = step(b)
    torch.cuda.synchronize()

    # ---- timed region (device-resident inputs) ----
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    recs = []
    infos = []
    e0.record(stream)
    for _ in range(args.steps):
        infos.append(step(b, recs))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    value, ms, total_bytes = replica_throughput(sum(step_bytes(i) for i in infos), ms, dist, dev)

    # per-solver breakdown from the in-step events
    names = ["spmv", "jacobi", "gauss_seidel", "cg", "bicgstab"]
    per = {k: [] for k in names}
    for ev in recs:
        for q, k in enumerate(names):
            per[k].append(ev[q].elapsed_time(ev[q + 1]))
    last = infos[-1]
    breakdown = {}
    for k in names:
        t_ms = statistics.median(per[k])
        its = 1 if k == "spmv" else last[k].iters
        gbs = BYTES[k] * N * its / (t_ms * 1e-3) / 1e9
        d = {"ms": round(t_ms, 4), "iters": its, "alg_GBps": round(gbs, 1)}
        if k != "spmv":
            d["status"] = last[k].status
            d["true_rel_res"] = last[k].true_rel_res
            if k in ("cg", "bicgstab"):
                d["time_to_tol_ms"] = round(t_ms, 4)
                d["us_per_iter"] = round(1e3 * t_ms / max(its, 1), 2)
            else:
                d["us_per_sweep"] = round(1e3 * t_ms / max(its, 1), 2)
        breakdown[k] = d

    # ---- roofline of the dominant kernel (largest share of the step) ----
    peak, peak_kind = load_peaks()
    fp64_meas = hs.fp64_rate() / 1e12      # TFLOP/s, measured on this GPU now
    roofline = None
    if not args.no_roofline:
        dom = max(["jacobi", "gauss_seidel", "cg", "bicgstab"], key=lambda k: statistics.median(per[k]))
        ra, rb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        dts, its = [], 0
        for _ in range(3):
            xs[dom].zero_()
            torch.cuda.synchronize()
            ra.record(stream)
            if dom == "cg":
                _, inf = hs.cg(A, b, xs["cg"], tol=args.tol, maxit=maxk, inplace=True, true_residual=False,
                               timeout_s=tmo)
            elif dom == "bicgstab":
                _, inf = hs.bicgstab(U, b, xs["bicgstab"], tol=args.tol, maxit=maxk, inplace=True,
                                     true_residual=False, timeout_s=tmo)
            elif dom == "jacobi":
                _, inf = hs.jacobi(A, b, xs["jacobi"], maxit=args.sweeps, inplace=True, true_residual=False,
                                   timeout_s=tmo)
            else:
                _, inf = hs.gauss_seidel(A, b, xs["gs"], maxit=args.sweeps, inplace=True, true_residual=False,
                                         timeout_s=tmo)
            rb.record(stream)
            torch.cuda.synchronize()
            dts.append(ra.elapsed_time(rb))
            its = inf.iters
        dt = statistics.median(dts)
        hbm_gbs = BYTES[dom] * N * its / (dt * 1e-3) / 1e9
        tflops = FLOPS[dom] * N * its / (dt * 1e-3) / 1e12
        clk = (clocks.get("sm_mhz") or 2070.0) * 1e6
        fp64_derived = FP64_FLOPS_PER_CLK * clk / 1e12
        kname = {"cg": "k_cg", "bicgstab": "k_bicgstab", "jacobi": "k_jacobi", "gauss_seidel": "k_gs"}[dom]
        roofline = {"kernel": kname + " (FP64, persistent: one launch per solve)", "bound": "alu",
                    "achieved": round(tflops, 4), "peak": round(fp64_meas, 4), "unit": "TFLOP/s",
                    "frac": round(tflops / fp64_meas, 4),
                    "peak_source": "measured: FP64 FMA rate of independent chains in every resident thread "
                                   "(hs_diag_fp64_rate), before the timed region",
                    "peak_derived": round(fp64_derived, 4),
                    "peak_derived_source": "2 FMA lanes/SM/clock x 2 flops x 152 SMs x %.0f MHz (median SM "
                                           "clock sampled in the timed region)" % (clk / 1e6),
                    "frac_of_derived": round(tflops / fp64_derived, 4),
                    "traffic": (round(TRAFFIC_B_PER_UNIT[dom] * N * its) if dom in TRAFFIC_B_PER_UNIT else None),
                    "traffic_source": "ncu DRAM bytes per unknown-iteration of a 10-iteration launch at 256^3 "
                                      "x N x iterations",
                    "flops_per_unknown_iter": FLOPS[dom], "iters": its, "launch_ms": round(dt, 3),
                    "hbm": {"achieved": round(hbm_gbs, 1), "peak": peak, "unit": "GB/s",
                            "frac": round(hbm_gbs / peak, 4), "peak_source": peak_kind,
                            "alg_bytes_per_unknown_iter": BYTES[dom]}}

    # ---- e2e: host buffers, copies inside the timed region ----
    e2e = None
    if not args.no_e2e:
        bp = torch.from_numpy(b_host).pin_memory()
        outs = {k: torch.empty(N, dtype=torch.float64).pin_memory() for k in xs}
        bd = torch.empty(N, dtype=torch.float64, device=dev)
        barrier()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_infos = []
        copy_stream = torch.cuda.Stream(dev)

        def start_copy(name):
            # the solution is final: copy it out on the side stream while the
            # next solver runs on the main one
            copy_stream.wait_stream(stream)
            with torch.cuda.stream(copy_stream):
                outs[name].copy_(xs[name], non_blocking=True)

        f0.record(stream)
        for _ in range(args.steps):
            stream.wait_stream(copy_stream)   # the previous step's copies read xs
            bd.copy_(bp, non_blocking=True)
            e_infos.append(step(bd, on_done=start_copy))
        stream.wait_stream(copy_stream)
        f1.record(stream)
        torch.cuda.synchronize()
        ems = f0.elapsed_time(f1)
        e_value, ems, _ = replica_throughput(sum(step_bytes(i) for i in e_infos), ems, dist, dev)
        e2e = {"value": e_value, "unit": "GB/s", "h2d_bytes_per_step": 8 * N,
               "d2h_bytes_per_step": 8 * N * len(xs), "ms_per_step": ems / args.steps}

    # ---- CPU baseline (rank 0, N = 1 only) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        nb1, secs1, desc1, _ = oracle_sample(n, b_host)
        nb, secs, desc, cores = oracle_sample(n, b_host, all_cores=True)
        cpu = {"value": nb / secs / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": desc,
               "seconds": round(secs, 2),
               "single_core": {"value": nb1 / secs1 / 1e9, "cores": 1, "seconds": round(secs1, 2)}}

    extras = {}
    if rank == 0 and args.mixed_n > 0:
        extras["mixed_vs_fp64"] = mixed_comparison(args.mixed_n, dev, tmo)
    if rank == 0 and args.adjoint_n > 0:
        extras["adjoint"] = adjoint_timing(args.adjoint_n, dev, tmo)
    if rank == 0 and args.batch_n > 0:
        extras["batched"] = batch_comparison(args.batch_n, dev, tmo, args.batch_vark)
    if rank == 0 and not args.no_variants:
        extras["paper_variants"] = variant_comparison(n, dev, tmo)
    if rank == 0 and args.hpcg_nz > 0:
        extras["hpcg"] = hpcg_timing(args.hpcg_nz, dev, tmo)
    if rank == 0 and not args.no_variants:
        extras["temporal_blocking"] = blocking_timing(n, args.sweeps, dev, tmo)
        extras["poisson2d"] = poisson2d_timing(dev, tmo)

    # kernels launched per step: spmv 1; jacobi, cg, bicgstab: control init +
    # persistent solver + residual + finalize = 4 each; gauss-seidel: solver +
    # residual + finalize = 3 (its control block is uploaded by a copy)
    launches_per_step = 1 + 4 + 3 + 4 + 4
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "poisson3d %d^3 FP64: SpMV + Jacobi x%d + lexicographic GS x%d + CG and "
                                   "BiCGStab(upwind, Pe 0.5) to %g" % (n, args.sweeps, args.sweeps, args.tol),
                       "grid": [n, n, n], "unknowns": N, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs and solver state (>= 2 x 134 MB per solver) exceed the 129 MB L2; no flush"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps, "clocks": clocks, "solvers": breakdown,
        }
        line.update(summaries(extras))
        line["extras"] = extras
        print(json.dumps(line), flush=True)


def summaries(extras):
    """Short top-level keys for the second half of the metric (time to 1e-10,
    mixed / batched against plain FP64); the extras hold the detail."""
    out = {}
    m = extras.get("mixed_vs_fp64")
    if m:
        out["mixed512"] = {"fp64_cg_s": round(m["fp64_cg"]["ms"] / 1e3, 3), "fp64_cg_iters": m["fp64_cg"]["iters"],
                           "mixed_s": round(m["mixed"]["ms"] / 1e3, 3), "outer": m["mixed"]["outer"],
                           "inner_iters": m["mixed"]["inner_iters"], "speedup": m["speedup"],
                           "mixed_true_rel_res": m["mixed"]["true_rel_res"],
                           "rel_err_vs_gpu_fp64_cg": m["mixed"]["rel_err_vs_fp64_solution"]}
        if "rel_err_vs_oracle_4096_cells" in m["mixed"]:
            out["mixed512"]["rel_err_vs_oracle"] = {"mixed": m["mixed"]["rel_err_vs_oracle_4096_cells"],
                                                    "fp64_cg": m["fp64_cg"]["rel_err_vs_oracle_4096_cells"],
                                                    "sample": "4096 seeded cells of the oracle's FP64 CG solution"}
    bt = extras.get("batched")
    if bt:
        out["batched512"] = {"fp64_s": round(bt["batched"]["ms"] / 1e3, 3),
                             "mixed_s": round(bt["batched_mixed"]["ms"] / 1e3, 3),
                             "sequential_fp64_s": round(bt["sequential"]["ms"] / 1e3, 3),
                             "speedup_fp64": bt["speedup"], "speedup_mixed": bt["speedup_mixed_vs_sequential"],
                             "converged": [bt["batched"]["converged"], bt["batched_mixed"]["converged"]]}
    ad = extras.get("adjoint")
    if ad:
        out["adjoint256"] = {"fp64_s": round(ad["fp64"]["ms_forward_adjoint_gradient"] / 1e3, 3),
                             "mixed_s": round(ad["mixed"]["ms_forward_adjoint_gradient"] / 1e3, 3)}
    return out


def poisson2d_timing(dev, tmo):
    """The small configuration (2-D Poisson, 128^2 interior nodes, FP64, b ~ U(-1,1)):
    Jacobi x500, lexicographic GS x500, CG and BiCGStab to 1e-10; the working set
    is L2-resident, so iterations/s and time-to-tolerance are the figures."""
    import torch

    import paper_2305_05988_gb300 as hs
    from paper_2305_05988_gb300 import inputs
    shape = (128, 128)
    A = hs.Operator.laplacian(shape)
    b = torch.from_numpy(inputs.rhs_uniform(shape, 0)).to(dev)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": "poisson2d 128^2 FP64: Jacobi x500, GS x500, CG and BiCGStab to 1e-10"}
    runs = (("jacobi", hs.jacobi, {"maxit": 500}), ("gauss_seidel", hs.gauss_seidel, {"maxit": 500}),
            ("cg", hs.cg, {"tol": 1e-10, "maxit": 20000}), ("bicgstab", hs.bicgstab, {"tol": 1e-10, "maxit": 20000}))
    for name, fn, kw in runs:
        fn(A, b, true_residual=False, timeout_s=max(tmo, 10.0), **kw)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        _, info = fn(A, b, true_residual=False, timeout_s=max(tmo, 10.0), **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"ms": round(ms, 3), "iters": info.iters, "iters_per_s": round(info.iters / (ms * 1e-3), 1)}
    return out


def blocking_timing(n, sweeps, dev, tmo):
    """Temporal blocking of Jacobi on the step's Laplacian: 1..4 sweeps per pass
    over the grid, FP64 and FP32, microseconds per sweep (the iterates are
    bitwise those of one sweep per pass)."""
    import torch

    import paper_2305_05988_gb300 as hs
    from paper_2305_05988_gb300 import inputs
    shape = (n, n, n)
    A = hs.Operator.laplacian(shape)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": "%d^3 Laplacian, Jacobi x%d, sweeps per pass 1..4" % (n, sweeps)}
    for dt, name in ((torch.float64, "f64"), (torch.float32, "f32")):
        b = torch.from_numpy(inputs.rhs_uniform(shape, 0)).to(device=dev, dtype=dt)
        rec = {}
        for spp in (1, 2, 3, 4):
            hs.jacobi(A, b, maxit=sweeps, sweeps_per_pass=spp, true_residual=False, timeout_s=max(tmo, 10.0))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            hs.jacobi(A, b, maxit=sweeps, sweeps_per_pass=spp, true_residual=False, timeout_s=max(tmo, 10.0))
            e1.record(stream)
            torch.cuda.synchronize()
            rec["spp%d" % spp] = round(1e3 * e0.elapsed_time(e1) / sweeps, 2)
        out[name + "_us_per_sweep"] = rec
        del b
    torch.cuda.empty_cache()
    return out


def hpcg_timing(nz, dev, tmo):
    """The paper's own benchmark system (section 4.1) on the grid of one of its
    nodes, 128 x 128 x nz (nz = 6144: 48 ranks of 128^3): HPCG's 7- and 27-point
    matrices (diagonal 27, -1 per neighbour), b = A 1, x0 = 0, absolute
    criterion ||r|| < 1e-6.  Time to criterion and per iteration for CG, CG-NB,
    BiCGStab and Jacobi, with the paper's printed iteration counts beside ours
    (its per-iteration times on a 48-core node are context, not a target)."""
    import torch

    import paper_2305_05988_gb300 as hs
    shape = (128, 128, nz)
    stream = torch.cuda.current_stream(dev)
    paper = {"hpcg7": {"cg": 12, "bicgstab": 8, "jacobi": 18}, "hpcg27": {"cg": 72, "bicgstab": 45, "jacobi": 515}}
    # the paper's wall times on one MareNostrum 4 node (2x Xeon Platinum 8160,
    # 48 cores, MPI-only, same grid): context, not a target
    paper_s = {"hpcg7": {"cg": 1.52, "bicgstab": 1.96, "jacobi": 1.40},
               "hpcg27": {"cg": 19.35, "bicgstab": 23.76, "jacobi": 113.91}}
    out = {"workload": "HPCG %dx%dx%d, b = A 1, x0 = 0, ||r|| < 1e-6" % shape}
    for pts in (7, 27):
        A = hs.Operator.hpcg(shape, pts)
        b = A.spmv(torch.ones(A.N, dtype=torch.float64, device=dev))
        tol = 1e-6 / torch.linalg.norm(b).item()
        rec = {}
        for name, fn in (("cg", hs.cg), ("cg_nb", hs.cg_nb), ("bicgstab", hs.bicgstab), ("jacobi", hs.jacobi)):
            fn(A, b, tol=tol, maxit=5000, history=False, true_residual=False, timeout_s=max(tmo, 10.0))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            x, info = fn(A, b, tol=tol, maxit=5000, history=False, true_residual=False, timeout_s=max(tmo, 10.0))
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            rec[name] = {"ms": round(ms, 3), "iters": info.iters, "paper_iters": paper["hpcg%d" % pts].get(name),
                         "paper_node_s": paper_s["hpcg%d" % pts].get(name),
                         "us_per_iter": round(1e3 * ms / max(info.iters, 1), 2), "status": info.status,
                         "max_err_vs_ones": torch.max(torch.abs(x - 1.0)).item()}
            del x
        # symmetric Gauss-Seidel (the paper's GS is symmetric but processor-local:
        # its counts are context).  A 27-point sweep is a chain through all
        # 6144 z planes (the plane-lagged kernel, about 11 us per plane), so it
        # is timed over two iterations rather than run to the criterion.
        gs_it = 5000 if pts == 7 else 2
        gs_tol = tol if pts == 7 else 0.0
        kw = dict(tol=gs_tol, maxit=gs_it, mode="symmetric", true_residual=False, timeout_s=max(tmo, 10.0))
        hs.gauss_seidel(A, b, **(kw if pts == 7 else dict(kw, maxit=1)))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        x, info = hs.gauss_seidel(A, b, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        rec["gauss_seidel_symmetric"] = {
            "ms": round(ms, 3), "iters": info.iters, "paper_iters": 9 if pts == 7 else 142,
            "us_per_iter": round(1e3 * ms / max(info.iters, 1), 2), "status": info.status,
            "run": "to the criterion" if pts == 7 else "2 iterations (per-iteration time only)"}
        del x
        out["hpcg%d" % pts] = rec
        del A, b
    torch.cuda.empty_cache()
    return out


def variant_comparison(n, dev, tmo):
    """The paper's proposed variants on the step's systems: CG-NB (Algorithm 1,
    one fused pass and one grid reduction per iteration) against classical CG
    on the Laplacian, and BiCGStab in Algorithm 2's order (B1) against the
    classical order on the upwind operator; time to 1e-10 and per iteration."""
    import torch

    import paper_2305_05988_gb300 as hs
    from paper_2305_05988_gb300 import inputs
    shape = (n, n, n)
    b = torch.from_numpy(inputs.rhs_uniform(shape, 0)).to(dev)
    A = hs.Operator.laplacian(shape)
    U = hs.Operator.upwind(shape, inputs.upwind_beta(shape, 0.5))
    stream = torch.cuda.current_stream(dev)
    out = {"workload": "%d^3: CG / CG-NB on the Laplacian, BiCGStab / B1 on upwind (Pe 0.5), tol 1e-10" % n}
    runs = (("cg", hs.cg, A, {}), ("cg_nb", hs.cg_nb, A, {}), ("bicgstab", hs.bicgstab, U, {}),
            ("bicgstab_b1", hs.bicgstab, U, {"paper_order": True}))
    for name, fn, op, kw in runs:
        fn(op, b, tol=1e-10, maxit=20000, history=False, true_residual=False, timeout_s=max(tmo, 10.0), **kw)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        x, info = fn(op, b, tol=1e-10, maxit=20000, history=False, true_residual=False,
                     timeout_s=max(tmo, 10.0), **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"ms": round(ms, 2), "iters": info.iters, "us_per_iter": round(1e3 * ms / max(info.iters, 1), 2),
                     "status": info.status, "true_rel_res": op.residual(b, x).norm().item() / b.norm().item()}
    out["cg_nb_speedup"] = round(out["cg"]["ms"] / out["cg_nb"]["ms"], 3)
    del b, A, U
    torch.cuda.empty_cache()
    return out


def mixed_comparison(n, dev, tmo):
    """Time-to-1e-10 on the variable-coefficient diffusion system (log k ~ N(0,1)):
    plain FP64 CG against FP32-inner / FP64-outer refinement on the same GPU."""
    import torch

    import paper_2305_05988_gb300 as hs
    from paper_2305_05988_gb300 import inputs
    shape = (n, n, n)
    k = torch.from_numpy(np.exp(inputs.log_k(shape, 1.0, 0))).to(dev)
    b = torch.from_numpy(inputs.rhs_uniform(shape, 0)).to(dev)
    A = hs.Operator.diffusion(shape, k)
    out = {"workload": "%d^3 diffusion, log k ~ N(0,1), f ~ U(-1,1), tol 1e-10" % n}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize()
    ev[0].record(stream)
    x, info = hs.cg(A, b, tol=1e-10, maxit=200000, history=False, timeout_s=max(tmo, 10.0))
    ev[1].record(stream)
    xm, im = hs.solve_mixed(A, b, tol=1e-10, maxit=40, inner_tol=1e-4, inner_maxit=200000,
                            timeout_s=max(tmo, 10.0))
    ev[2].record(stream)
    torch.cuda.synchronize()
    t64 = ev[0].elapsed_time(ev[1])
    tmx = ev[1].elapsed_time(ev[2])
    err = (torch.linalg.norm(xm - x) / torch.linalg.norm(x)).item()
    out["fp64_cg"] = {"ms": round(t64, 2), "iters": info.iters, "true_rel_res": info.true_rel_res,
                      "status": info.status}
    out["mixed"] = {"ms": round(tmx, 2), "outer": im.outer, "inner_iters": im.inner_iters,
                    "true_rel_res": im.true_rel_res, "status": im.status, "inner_tol": 1e-4,
                    "rel_err_vs_fp64_solution": err}
    out["speedup"] = round(t64 / tmx, 3)
    # error against the FP64 oracle's own solution of this system, sampled at
    # the cells stored by tests/golden/make_mixed512.py (512^3 only)
    gold_path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "mixed512_solution.json")
    if n == 512 and os.path.exists(gold_path):
        with open(gold_path) as fh:
            gold = json.load(fh)
        cells = torch.tensor(gold["cells"], dtype=torch.long, device=dev)
        ref = torch.tensor(gold["x_at_cells"], dtype=torch.float64, device=dev)
        rn = torch.linalg.norm(ref).item()
        out["fp64_cg"]["rel_err_vs_oracle_4096_cells"] = (torch.linalg.norm(x[cells] - ref) / rn).item()
        out["mixed"]["rel_err_vs_oracle_4096_cells"] = (torch.linalg.norm(xm[cells] - ref) / rn).item()
    del A, k, b, x, xm
    torch.cuda.empty_cache()
    return out


def adjoint_timing(n, dev, tmo):
    """Forward solve, adjoint solve and per-cell gradient of L = ||u - u_obs||^2
    on the 256^3 inverse-diffusion workload (log k ~ N(0, 0.5^2))."""
    import torch

    import paper_2305_05988_gb300 as hs
    from paper_2305_05988_gb300 import inputs
    shape = (n, n, n)
    logk = torch.from_numpy(inputs.log_k(shape, 0.5, 0)).to(dev).requires_grad_(True)
    f = torch.from_numpy(inputs.rhs_uniform(shape, 0)).to(dev).requires_grad_(True)
    k2 = hs.exp_logk(torch.from_numpy(inputs.log_k(shape, 0.5, 0, inputs.STREAM_K2)).to(dev))
    u_obs = hs.cg(hs.Operator.diffusion(shape, k2), f.detach(), tol=1e-12, maxit=200000, history=False,
                  timeout_s=max(tmo, 10.0))[0]
    stream = torch.cuda.current_stream(dev)
    out = {"workload": "%d^3 inverse diffusion, log k ~ N(0, 0.5^2), tol 1e-10" % n}
    # warm-up on a 16^3 problem: the first autograd pass loads torch's own
    # kernels (seconds, once per process), which is not the solve's time
    ws = (16, 16, 16)
    lw = torch.from_numpy(inputs.log_k(ws, 0.5, 0)).to(dev).requires_grad_(True)
    fw = torch.from_numpy(inputs.rhs_uniform(ws, 0)).to(dev).requires_grad_(True)
    for mixed in (False, True):
        uw = hs.diffusion_solve(lw, fw, ws, tol=1e-10, mixed=mixed, maxit=200000)
        torch.sum((uw - 0.5 * uw.detach()) ** 2).backward()
    torch.cuda.synchronize()
    for mixed in (False, True):
        logk.grad = None
        f.grad = None
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        u = hs.diffusion_solve(logk, f, shape, tol=1e-10, mixed=mixed, maxit=200000)
        L = torch.sum((u - u_obs) ** 2)
        L.backward()
        e1.record(stream)
        torch.cuda.synchronize()
        out["mixed" if mixed else "fp64"] = {"ms_forward_adjoint_gradient": round(e0.elapsed_time(e1), 2),
                                             "loss": L.item(),
                                             "grad_logk_norm": torch.linalg.norm(logk.grad).item()}
    del logk, f, k2, u_obs
    torch.cuda.empty_cache()
    return out


def batch_comparison(nsys, dev, tmo, vark=False):
    """The batched workload: nsys independent systems (2-D or 3-D, sides
    log-uniform in [16, 256]; even systems CG on the symmetric diffusion
    operator (k = 1, or log k ~ N(0, 1) with vark), odd systems BiCGStab on
    upwind convection-diffusion with Peclet in [0.1, 1]) solved to 1e-8 by one
    persistent kernel replayed as a CUDA graph: in FP64, and in mixed precision
    (FP64 refinement, FP32 inner CG / BiCGStab to 1e-4), against solving them
    one after another with the standalone FP64 solvers."""
    import torch

    import paper_2305_05988_gb300 as hs
    from paper_2305_05988_gb300 import inputs
    systems = inputs.batch_systems(nsys, seed=0)
    ops, bs, sol, ks = [], [], [], []
    for s in systems:
        if s.solver == "cg" and vark:
            k = torch.from_numpy(np.exp(inputs.log_k(s.shape, 1.0, s.index))).to(dev)
            ks.append(k)
            ops.append(hs.Operator.diffusion(s.shape, k))
        elif s.solver == "cg":
            ops.append(hs.Operator.laplacian(s.shape))
        else:
            ops.append(hs.Operator.upwind(s.shape, inputs.upwind_beta(s.shape, s.peclet)))
        bs.append(torch.from_numpy(inputs.uniform_pm1(0, inputs.STREAM_BATCH_RHS + s.index, s.N)).to(dev))
        sol.append(s.solver)
    unknowns = sum(s.N for s in systems)
    st = torch.cuda.Stream(dev)
    out = {"workload": "%d systems, sides log-uniform in [16, 256], 2-D/3-D, CG (%s) / BiCGStab "
                       "(upwind, Pe in [0.1, 1]), tol 1e-8" % (nsys, "diffusion, log k ~ N(0,1)" if vark else "Laplacian"),
           "unknowns": unknowns}
    t0 = time.perf_counter()
    batch = hs.Batch(ops, sol, autotune=True)
    out["autotune_s"] = round(time.perf_counter() - t0, 2)
    with torch.cuda.stream(st):
        xs = [torch.zeros_like(b) for b in bs]
        batch.solve(bs, xs, tol=1e-8, timeout_s=max(tmo, 20.0))   # warm-up: captures the graph
        for x in xs:
            x.zero_()
        st.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(st)
        xs, infos = batch.solve(bs, xs, tol=1e-8, timeout_s=max(tmo, 20.0))
        e1.record(st)
        seq_iters = 0
        for A, b, s in zip(ops, bs, sol):
            fn = hs.cg if s == "cg" else hs.bicgstab
            _, info = fn(A, b, tol=1e-8, history=False, true_residual=False, timeout_s=max(tmo, 10.0))
            seq_iters += info.iters
        e2.record(st)
        st.synchronize()
    tb, ts = e0.elapsed_time(e1), e1.elapsed_time(e2)
    out["batched"] = {"ms": round(tb, 2), "graph": batch.graph_used, "iters_total": sum(i.iters for i in infos),
                      "converged": sum(i.status == "OK" for i in infos), "teams_gt1": sum(t > 1 for t in batch.teams)}
    out["sequential"] = {"ms": round(ts, 2), "iters_total": seq_iters}
    out["speedup"] = round(ts / tb, 3)
    del batch
    # mixed precision: the same systems, FP64 refinement with FP32 inner solves
    mb = hs.Batch(ops, ["mixed"] * len(ops), autotune=True)
    with torch.cuda.stream(st):
        for x in xs:
            x.zero_()
        mb.solve(bs, xs, tol=1e-8, maxit=20, inner_tol=1e-4, inner_maxit=100000, timeout_s=max(tmo, 20.0))
        for x in xs:
            x.zero_()
        st.synchronize()
        e0.record(st)
        xs, minfo = mb.solve(bs, xs, tol=1e-8, maxit=20, inner_tol=1e-4, inner_maxit=100000,
                             timeout_s=max(tmo, 20.0))
        e1.record(st)
        st.synchronize()
    tm = e0.elapsed_time(e1)
    out["batched_mixed"] = {"ms": round(tm, 2), "graph": mb.graph_used,
                            "outer_total": sum(i.outer for i in minfo),
                            "inner_iters_total": sum(i.inner_iters for i in minfo),
                            "converged": sum(i.status == "OK" for i in minfo),
                            "max_rel_res": max(i.rel_res for i in minfo)}
    out["speedup_mixed_vs_sequential"] = round(ts / tm, 3)
    del mb, xs, bs, ops, ks
    torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "ours" and world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
