#!/usr/bin/env python3
"""Throughput of the PinT-QBVM / PinT-MQBVM all-at-once direct solve on GB300.

Workload (default): 2D unit square, 255^2 interior points (5-point Laplacian),
256 time levels, T = 0.1 -- 16 646 400 all-at-once unknowns per solve -- with
z(., 0) a sum of 16 random decaying sine modes and g_delta the discrete forward
solution plus 1% Gaussian noise (seeded).  One step solves BOTH formulations
(PinT-QBVM with alpha = delta, PinT-MQBVM with alpha = tau*delta, the a-priori
rule of Section 5): 2 x 16 646 400 unknowns.  The right-hand side is given in
full ("general": f_h of eq. 3.3/3.6 with every level stored and read), or as g
only ("delta", --rhs delta).

Metric: all-at-once unknowns solved per second (whole job, all ranks).  The
device-timed value uses CUDA events around each step on the solve stream with
the inputs resident in HBM and an L2 flush (a 256 MB write) between steps
outside the timed events.  e2e repeats the step through the same C ABI with
pinned HOST buffers, so the host<->device copies are inside the timing.

  python bench.py [--gpus N --steps K --warmup W] [--rhs general|delta]
  python bench.py --impl reference ...     # the CPU FP64 oracle, timed alone
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "all-at-once unknowns solved/sec and HBM GB/s fraction at <=1e-10 rel err vs FP64 oracle"
UNIT = "unknowns/s"
# FP64 ALU peak derived from the part's unit counts and clock (152 SMs x 2 FP64
# operations per clock x 2.07 GHz): context only; the roofline uses the rate
# qbvm_measure_peak measures in the run.
FP64_PEAK_DERIVED_TOPS = 152 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + write) per launch of the headline kernels from one ncu
# capture, valid only for the kernel sources whose hash is stored beside them
# (traffic_source_hash()); any change to the sources makes them stale (null).
PROFILED_TRAFFIC = {"sources": "9d664fb8f4c5cf15",
                    "bytes": {"dst_x": 211369216, "dst_y": 210454272, "time_solve": 355708160}}


TRAFFIC_SOURCES = ("qbvm_dst.cuh", "qbvm_fft.cuh", "qbvm_timesolve.cuh")


def traffic_source_hash() -> str:
    """Hash of the sources of the headline's FP64 DST-I and time-solve tiles
    (the kernels whose DRAM traffic PROFILED_TRAFFIC records)."""
    import hashlib
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2107_06381_gb300", "csrc")
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def flop_budget(name, grid):
    """Algorithmic FP64 flops of one launch by the per-element counts of the
    path's flop budget: a DST-I pass ~22 flops per element; the time solve
    2 x 5 log2(nt) (FFT + inverse FFT) + ~11 (Step (b) divide) + ~10 (omega
    scaling and unscaling) per element."""
    units = grid.nt * grid.Nx
    if name.startswith("dst_"):
        return 22.0 * units
    if name == "time_solve":
        return (10.0 * math.log2(grid.nt) + 21.0) * units
    return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--rhs", choices=["general", "delta"], default="general")
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-refine", action="store_true", help="skip the FP32+refinement variant")
    ap.add_argument("--refine-only", action="store_true",
                    help="profiling aid: run only the FP32+refinement variant (no JSON headline)")
    ap.add_argument("--c5", action="store_true",
                    help="only the learned-alpha workload at its full size (200k labelled 2D 127^2 x 128 "
                         "instances, 4096 held out); several minutes")
    ap.add_argument("--leg", choices=["c3_3d", "c4_sweep", "c4_full_multi", "c1_batched", "batched_2d",
                                      "learned_alpha"],
                    help="run one of the secondary workloads alone (its JSON object only, no headline)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the 3D (127^3 x 128) and batched-sweep (512 instances) measurements")
    return ap.parse_args()


def workload():
    import bhcp_inputs as bi
    return bi.make_c2()


def _cores_used() -> int:
    try:
        from threadpoolctl import threadpool_info
        n = max((i.get("num_threads", 1) for i in threadpool_info()), default=1)
        return int(n)
    except Exception:
        return os.cpu_count() or 1


def cpu_oracle_leg(prob, forms, steps):
    """Time the CPU FP64 oracle (exact sine-basis solve) as it stands on the
    host cores; returns (unknowns/s, seconds list, solutions by form)."""
    import numpy as np
    import oracle as O
    grid = prob.grid
    times, sols = [], {}
    for i in range(steps):
        form = forms[i % len(forms)]
        alpha = O.alpha_apriori(form, prob.delta, grid.tau)
        F = O.delta_rhs(grid, form, alpha, prob.g_delta)
        t0 = time.perf_counter()
        y = O.solve_spectral(grid, form, alpha, F)
        times.append(time.perf_counter() - t0)
        sols[form] = y
    return grid.unknowns / statistics.median(times), times, sols


def cpu_oracle_one_core(timeout_s=180):
    """One full solve of the 2D workload by the oracle on ONE host core (for the
    comparison with a serial code): a child process with every BLAS / OpenMP
    thread count set to 1 before numpy loads.  Returns seconds, or None."""
    import subprocess
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[v] = "1"
    code = ("import time, bhcp_inputs as bi, oracle as O\n"
            "p = bi.make_c2(); a = O.alpha_apriori(O.PQ, p.delta, p.grid.tau)\n"
            "F = O.delta_rhs(p.grid, O.PQ, a, p.g_delta)\n"
            "t = time.perf_counter(); O.solve_spectral(p.grid, O.PQ, a, F); print(time.perf_counter() - t)\n")
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=timeout_s)
        return float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
    except Exception:
        return None


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- our arm

def _fft_ops(lm: int) -> float:
    """FP64 operations per complex element of the radix-4/2 Stockham FFT of
    length 2^lm: 4 per element in the first radix-4 pass (16 adds per
    butterfly), 6 in later radix-4 passes (four fused twiddle butterflies of 6
    operations, with w3 = w1 w2 factored out), 3 in the closing radix-2 pass
    (one fused twiddle butterfly)."""
    if lm == 0:
        return 0.0
    r4, r2 = lm // 2, lm % 2
    return (4.0 + 6.0 * (r4 - 1) if r4 else 0.0) + 3.0 * r2


def kernel_model(name, grid, rhs):
    """Algorithmic HBM bytes and FP64 operations (DADD, DMUL, DFMA count one each)
    of one launch of `name` in a full solve, from the kernels' arithmetic:

    time_solve, per real element: 2 (omega-scaling, rho^H folded into the
      table) + 2 x FFT(nt/2)/2 + 2 (one complex product by the plan's table
      cnorm / (d_k + tau Lambda_l), read as 8 more bytes) + 2 (unscaling).
    dst (length M per real column; the FP64 passes compute 4x the DST), per
      real element: 2 (pair pre-processing, one fused multiply-add each)
      + FFT(M)/2 + 1 (column separation) + 1 (prefix sum).
    Bytes: each pass reads and writes every FP64 value once."""
    nt, Nx = grid.nt, grid.Nx
    if name == "time_solve":
        reads = Nx if rhs == "delta" else nt * Nx
        byts = 8 * (reads + nt * Nx) + 16 * (nt // 2) * Nx
        ops = (2.0 + _fft_ops(int(math.log2(nt // 2))) + 2.0 + 2.0) * nt * Nx
        return byts, ops
    if name.startswith("dst_"):
        ax = "xyz".index(name[-1])
        M = grid.M[ax]
        byts = 16 * nt * Nx
        ops = (2.0 + _fft_ops(int(math.log2(M))) / 2 + 1.0 + 1.0) * nt * Nx
        return byts, ops
    return None, None


def measured_fp64_peak(device, stream):
    """FP64 FMA rate of this GPU measured now (qbvm_measure_peak), with the
    median SM clock nvidia-smi saw while the probe ran."""
    import paper_2107_06381_gb300 as Q
    sampler = ClockSampler(device.index if device.index is not None else 0)
    sampler.start()
    time.sleep(0.1)
    rate = 0.0
    for _ in range(4):              # ~0.1 s of probe launches under the sampler
        rate = max(rate, Q.qbvm_measure_peak(Q.PEAK_FP64_FMA, stream=stream))
    clocks = sampler.stop()
    return rate, clocks


def roofline(kstats, grid, rhs, value, device, stream):
    """Roofline object of the dominant kernel of the headline step.

    bound "alu": the FP64 pipe, against the DFMA rate measured in this run;
    `frac` counts the kernel's own FP64 instructions (DADD, DMUL, DFMA one
    each, kernel_model).  Beside it: the same launch by the path's flop budget
    (flop_budget, over twice the FMA rate), and the HBM fraction of its
    algorithmic bytes over the measured copy peak."""
    hbm_peak, hbm_src = _peaks()
    dname, (dl, dms) = max(kstats.items(), key=lambda kv: kv[1][1])
    byts, ops = kernel_model(dname, grid, rhs)
    if byts is None:
        return {"kernel": dname, "note": "no model for this kernel"}
    avg_s = dms / dl / 1e3
    fma_rate, pclk = measured_fp64_peak(device, stream)
    peak_tops = fma_rate / 1e12
    src_hash = traffic_source_hash()
    stale = PROFILED_TRAFFIC["sources"] != src_hash
    traffic = None if stale else PROFILED_TRAFFIC["bytes"].get(dname)
    t_hbm = byts / (hbm_peak * 1e9)
    t_alu = ops / fma_rate
    ach_ops = ops / avg_s / 1e12
    hbm_ach = byts / avg_s / 1e9
    fl = flop_budget(dname, grid)
    roof = {"bound": "alu" if t_alu > t_hbm else "hbm", "kernel": dname,
            "launches_traced": dl, "avg_ms": round(dms / dl, 4)}
    if t_alu > t_hbm:
        roof.update({"achieved": round(ach_ops, 4), "peak": round(peak_tops, 4),
                     "unit": "T FP64-op/s (DADD/DMUL/DFMA = 1 op)", "frac": round(ach_ops / peak_tops, 4)})
    else:
        roof.update({"achieved": round(hbm_ach, 1), "peak": hbm_peak, "unit": "GB/s",
                     "frac": round(hbm_ach / hbm_peak, 4)})
    bpu = 16 if rhs == "general" else 8
    roof.update({
        "peak_source": "measured in-run: qbvm_measure_peak (independent DFMA chains on every SM, best of 5)",
        "fp64_fma_per_s_measured": fma_rate,
        "fp64_peak_sm_mhz": pclk.get("sm_mhz"),
        "fp64_peak_derived_tops": round(FP64_PEAK_DERIVED_TOPS, 4),
        "fractions": {
            "fp64_ops_of_measured": round(ach_ops / peak_tops, 4),
            "flop_budget_of_measured": round(fl / avg_s / (2 * fma_rate), 4) if fl else None,
            "hbm_algorithmic_of_measured": round(hbm_ach / hbm_peak, 4),
        },
        "kernel_fp64_ops_per_launch": ops, "flop_budget_per_launch": fl,
        "algorithmic_bytes_per_launch": byts,
        "hbm_achieved_gbs": round(hbm_ach, 1), "hbm_peak_gbs": hbm_peak, "hbm_peak_source": hbm_src,
        "traffic": traffic,
        "traffic_note": ("stale: the kernel sources changed since the ncu capture" if stale
                         else "dram__bytes_read.sum + dram__bytes_write.sum per launch, ncu"),
        "dram_gbs_ncu": round(traffic / avg_s / 1e9, 1) if traffic else None,
        "solve_algorithmic_gbs": round(bpu * value / 1e9, 1),
        "solve_algorithmic_frac": round(bpu * value / 1e9 / hbm_peak, 4),
    })
    return roof


def our_arm(args, rank, world, device):
    import numpy as np
    import torch
    import paper_2107_06381_gb300 as Q

    Q.build_library()
    Q.load_library()
    prob = workload()
    grid = prob.grid
    forms = [Q.FORM_PQ, Q.FORM_PM]
    rhs_kind = Q.RHS_GENERAL if args.rhs == "general" else Q.RHS_DELTA
    stream = torch.cuda.Stream(device)
    plans, inputs, outputs = [], [], []
    for form in forms:
        alpha = prob.delta if form == Q.FORM_PQ else grid.tau * prob.delta
        plans.append(Q.Plan(grid.dim, grid.M, grid.L, grid.T, grid.nt, form, alpha, 0.0, Q.FP64, rhs_kind))
        if rhs_kind == Q.RHS_GENERAL:
            # f_h of eq. 3.3 / 3.6 stored in full: level 0 = -omega g / tau, others 0
            omega = -1.0 / alpha if form == Q.FORM_PQ else -grid.tau / alpha
            F = np.zeros(grid.full_shape)
            F[0] = -omega / grid.tau * prob.g_delta
        else:
            F = prob.g_delta
        inputs.append(torch.as_tensor(np.ascontiguousarray(F).ravel(), dtype=torch.float64, device=device))
        outputs.append(torch.empty(grid.unknowns, dtype=torch.float64, device=device))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)    # 256 MB > L2

    def step():
        for plan, fin, yout in zip(plans, inputs, outputs):
            plan.solve(fin, yout, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(0 if args.refine_only else args.warmup):
            step()
    torch.cuda.synchronize(device)

    # ---- timed region (no per-kernel tracing inside it)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(device.index if device.index is not None else 0)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(device)
    sampler.start()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            evs[i][0].record(stream)
            if not args.refine_only:
                step()
            evs[i][1].record(stream)
            flush.zero_()                      # L2 flush between steps, outside the events
    torch.cuda.synchronize(device)
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    if world > 1:
        from paper_2107_06381_gb300.replicas import max_over_ranks
        total_ms = max_over_ranks(total_ms, device)
        torch.distributed.barrier()
    launches_per_solve = plans[0].info.kernels_per_solve
    unknowns_step = grid.unknowns * len(forms)
    value = world * unknowns_step * args.steps / (total_ms / 1e3) if total_ms > 0 else 0.0

    # ---- per-kernel times from a separate traced pass (CUDA events around
    # every kernel), after the timed region so that they do not perturb it
    kstats = {}
    if not args.refine_only:
        for plan in plans:
            plan.profile(True)
        with torch.cuda.stream(stream):
            for _ in range(max(3, args.steps // 4)):
                step()
                flush.zero_()
        torch.cuda.synchronize(device)
        for plan in plans:
            for name, (launches, ms) in plan.profile_read().items():
                a, b = kstats.get(name, (0, 0.0))
                kstats[name] = (a + launches, b + ms)
            plan.profile(False)

    # ---- roofline of the dominant kernel
    roof = roofline(kstats, grid, args.rhs, value, device, stream) if kstats else None
    kernels = {k: {"launches": v[0], "avg_ms": round(v[1] / v[0], 4), "share": round(v[1] / sum(x[1] for x in kstats.values()), 4)}
               for k, v in sorted(kstats.items(), key=lambda kv: -kv[1][1])} if kstats else {}

    # ---- FP32 transforms + FP64 refinement on the same inputs (reported beside the FP64 line)
    refine = None
    if not args.no_refine:
        rplans = []
        for form in forms:
            alpha = prob.delta if form == Q.FORM_PQ else grid.tau * prob.delta
            rplans.append(Q.Plan(grid.dim, grid.M, grid.L, grid.T, grid.nt, form, alpha, 0.0, Q.FP32_REFINE,
                                 rhs_kind))
        routs = [torch.empty_like(y) for y in outputs]

        def rstep():
            for plan, fin, yout in zip(rplans, inputs, routs):
                plan.solve(fin, yout, stream=stream)

        with torch.cuda.stream(stream):
            for _ in range(max(1, args.warmup)):
                rstep()
        torch.cuda.synchronize(device)
        revs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                revs[i][0].record(stream)
                rstep()
                revs[i][1].record(stream)
                flush.zero_()
        torch.cuda.synchronize(device)
        r_ms = sum(a.elapsed_time(b) for a, b in revs)
        # per-kernel times: a separate traced pass
        for plan in rplans:
            plan.profile(True)
        with torch.cuda.stream(stream):
            for _ in range(max(2, args.steps // 4)):
                rstep()
                flush.zero_()
        torch.cuda.synchronize(device)
        rk = {}
        for plan in rplans:
            for name, (launches, ms) in plan.profile_read().items():
                a, b = rk.get(name, (0, 0.0))
                rk[name] = (a + launches, b + ms)
            plan.profile(False)
        refine = {"value": world * unknowns_step * args.steps / (r_ms / 1e3), "unit": UNIT,
                  "ms_per_step": r_ms / args.steps, "dtype": "f32 transforms + double-float residual/update",
                  "refine_steps": [plan.info.last_refine_iters for plan in rplans],
                  "rel_residual": [plan.info.last_rel_residual for plan in rplans],
                  "kernels": {k: {"launches": v[0], "avg_ms": round(v[1] / v[0], 4)} for k, v in rk.items()},
                  "gpu_launches": sum(plan.info.kernels_per_solve for plan in rplans) * args.steps}
        for plan in rplans:
            plan.close()

    # ---- y^0 only from the delta right-hand side (a separate metric: the
    # forward time transform of f^0 e_0 is constant, so Step (c) at t = 0 is one
    # factor per spatial mode; DSTs of one level around it)
    y0m = None
    if not args.refine_only:
        y0plans = []
        for form in forms:
            alpha = prob.delta if form == Q.FORM_PQ else grid.tau * prob.delta
            y0plans.append(Q.Plan(grid.dim, grid.M, grid.L, grid.T, grid.nt, form, alpha, 0.0, Q.FP64, Q.RHS_DELTA))
        gdev = torch.as_tensor(np.ascontiguousarray(prob.g_delta).ravel(), dtype=torch.float64, device=device)
        y0s = [torch.empty(grid.Nx, dtype=torch.float64, device=device) for _ in forms]
        with torch.cuda.stream(stream):
            for plan, yo in zip(y0plans, y0s):
                plan.solve(gdev, yo, n0_only=True, stream=stream)
        torch.cuda.synchronize(device)
        nrep = 20
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(nrep):
                for plan, yo in zip(y0plans, y0s):
                    plan.solve(gdev, yo, n0_only=True, stream=stream)
            ev1.record(stream)
        torch.cuda.synchronize(device)
        ms = ev0.elapsed_time(ev1) / (nrep * len(forms))
        # against level 0 of the full delta-RHS solve
        yfull = torch.empty(grid.unknowns, dtype=torch.float64, device=device)
        y0plans[0].solve(gdev, yfull, stream=stream)
        torch.cuda.synchronize(device)
        diff = float((y0s[0] - yfull[:grid.Nx]).norm() / yfull[:grid.Nx].norm())
        y0m = {"metric": "y0-only solves/sec, delta right-hand side (a separate metric, not the headline)",
               "value": 1e3 / ms, "unit": "solves/s", "ms_per_solve": round(ms, 4),
               "outputs_per_solve": grid.Nx, "rel_diff_vs_full_solve_level0": diff,
               "kernels_per_solve": y0plans[0].info.kernels_per_solve}
        for plan in y0plans:
            plan.close()

    # ---- end to end through the C ABI with pinned host buffers
    host_in = [torch.empty(x.numel(), dtype=torch.float64, pin_memory=True) for x in inputs]
    host_out = [torch.empty(y.numel(), dtype=torch.float64, pin_memory=True) for y in outputs]
    for h, d in zip(host_in, inputs):
        h.copy_(d.cpu())
    for plan, hi, ho in zip(plans, host_in, host_out):     # warm-up (staging buffers)
        Q.qbvm_solve(plan.handle, hi.data_ptr(), ho.data_ptr(), False, stream.cuda_stream)
    e2e_times = []
    for _ in range(max(1, args.e2e_steps)):
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for plan, hi, ho in zip(plans, host_in, host_out):
            Q.qbvm_solve(plan.handle, hi.data_ptr(), ho.data_ptr(), False, stream.cuda_stream)
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = sum(e2e_times)
    if world > 1:
        from paper_2107_06381_gb300.replicas import max_over_ranks
        e2e_s = max_over_ranks(e2e_s, device)
    e2e = {"value": world * unknowns_step * len(e2e_times) / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": sum(x.numel() * 8 for x in inputs),
           "d2h_bytes_per_step": sum(y.numel() * 8 for y in outputs),
           "ms_per_step": round(1e3 * e2e_s / len(e2e_times), 3)}
    # the e2e outputs must equal the device-path outputs
    torch.cuda.synchronize(device)
    e2e_match = all(torch.equal(ho, y.cpu()) for ho, y in zip(host_out, outputs))

    # ---- CPU oracle leg (rank 0, N = 1) and accuracy of this run
    cpu = None
    rel_err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_oracle_leg(prob, forms[:1], 1)                  # warm-up (BLAS threads, page faults)
        cpu_val, cpu_times, sols = cpu_oracle_leg(prob, forms, 6)
        cpu = {"value": cpu_val, "unit": UNIT, "cores": _cores_used(), "kind": "oracle",
               "sample": "six full 255^2 x 256 solves, three per formulation (PinT-QBVM, PinT-MQBVM), by the "
                         "FP64 sine-basis oracle (dense DST-I matrices + exact per-mode recurrence) after one "
                         "warm-up solve; median",
               "seconds": [round(t, 3) for t in cpu_times]}
        one = cpu_oracle_one_core()
        if one:
            cpu["one_core"] = {"value": grid.unknowns / one, "unit": UNIT, "cores": 1, "seconds": round(one, 3),
                               "sample": "one full solve (PinT-QBVM), BLAS / OpenMP limited to one thread"}
        def max_err(ys):
            errs = []
            for form, y in zip(forms, ys):
                got = y.cpu().numpy()
                want = sols[form].ravel()
                errs.append(float(np.linalg.norm(got - want) / np.linalg.norm(want)))
            return max(errs)
        rel_err = max_err(outputs)
        if refine is not None:
            refine["rel_err_vs_oracle"] = max_err(routs)

    extra = {}
    if not args.no_extra and not args.refine_only:
        extra = run_legs(args, device, stream, flush, rank == 0 and world == 1 and not args.no_cpu_baseline)


    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": headline_config(args, grid, len(forms), f"replicas{world}"),
        "roofline": roof,
        "kernels": kernels,
        "e2e": e2e,
        "e2e_matches_device_path": e2e_match,
        "gpu_launches": launches_per_solve * len(forms) * args.steps,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "rel_err_vs_oracle": rel_err,
        "fp32_refine": refine,
        "y0_delta_rhs": y0m,
        **extra,
    }
    if args.refine_only:
        # profiling aid: the FP64 leg did not run, so it has no numbers
        out.update({"value": None, "ms_per_step": None, "roofline": None, "kernels": {}, "e2e": None,
                    "e2e_matches_device_path": None, "gpu_launches": refine["gpu_launches"] if refine else 0,
                    "note": "--refine-only: only the FP32 + refinement leg ran (fp32_refine)"})
    for plan in plans:
        plan.close()
    return out


def headline_config(args, grid, solves_per_step, parallelism):
    """The `config` of the headline line; the reference arm carries the same
    keys (its step solves one formulation at a time, alternating)."""
    return {"workload": f"c2_2d_255sq_x256_{args.rhs}_rhs", "dim": 2, "interior": [255, 255], "nt": 256,
            "T": grid.T, "forms": ["pint-qbvm", "pint-mqbvm"], "rhs": args.rhs,
            "unknowns_per_solve": grid.unknowns, "solves_per_step": solves_per_step,
            "l2": "flushed between steps (256 MB write outside the timed events); inputs 133 MB/solve",
            "parallelism": parallelism}


# ------------------------------------------------- 3D and batched-sweep rows

def _time_solves(plan, fin, yout, stream, steps, flush):
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        plan.solve(fin, yout, stream=stream)                 # warm-up
        for i in range(steps):
            evs[i][0].record(stream)
            plan.solve(fin, yout, stream=stream)
            evs[i][1].record(stream)
            flush.zero_()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / steps


def c3_leg(args, device, stream, flush, with_oracle):
    """3D unit cube, 127^3 interior points x 128 levels (262 M unknowns), delta
    right-hand side from 8 Gaussian bumps + 0.1% noise: the plain FP64 path
    against FP32 transforms with double-float refinement."""
    import numpy as np
    import torch
    import bhcp_inputs as bi
    import paper_2107_06381_gb300 as Q
    p = bi.make_c3()
    grid = p.grid
    alpha = p.delta
    g = torch.as_tensor(p.g_delta.ravel(), dtype=torch.float64, device=device)
    out = {"workload": "c3_3d_127cube_x128_delta_rhs", "unknowns": grid.unknowns}
    ys = {}
    for name, prec in (("fp64", Q.FP64), ("fp32_refine", Q.FP32_REFINE)):
        y = torch.empty(grid.unknowns, dtype=torch.float64, device=device)
        with Q.Plan(3, grid.M, grid.L, grid.T, grid.nt, Q.FORM_PQ, alpha, 0.0, prec, Q.RHS_DELTA) as plan:
            ms = _time_solves(plan, g, y, stream, max(2, args.steps // 5), flush)
            info = plan.info
            out[name] = {"ms_per_solve": ms, "value": grid.unknowns / (ms / 1e3), "unit": UNIT,
                         "refine_steps": info.last_refine_iters if prec == Q.FP32_REFINE else 0,
                         "rel_residual": info.last_rel_residual if prec == Q.FP32_REFINE else None}
        ys[name] = y
    if with_oracle:
        import oracle as O
        levels = [0, 1, 64, 127]
        want = O.solve_spectral(grid, O.PQ, alpha, O.rhs_block0(O.PQ, alpha, grid.tau, p.g_delta), levels=levels)
        for name, y in ys.items():
            got = y.view(grid.full_shape)[levels].cpu().numpy()
            out[name]["rel_err_vs_oracle_sampled_levels"] = O.rel_l2(got, want)
    return out


def c4_leg(args, device, stream, with_oracle=True):
    """512 uneven instances (1D n in {63..2047}, 2D {63,127,255}^2, nt in {32..512},
    relative noise log-uniform in [1e-4, 1e-2]) x 16 alphas, one persistent
    launch per run from a captured CUDA graph, launch shape autotuned.  The
    FP32 mode scans alpha in FP32 and sums y^0 at the picked alpha in
    double-float; the FP64 mode sums both in double-float (its DSTs in FP64).  With the oracle: the
    discrepancies of the four smallest instances at all 16 alphas, the pick,
    and y^0 at the pick, against the oracle's full solves."""
    import numpy as np
    import torch
    import bhcp_inputs as bi
    import paper_2107_06381_gb300 as Q
    specs = bi.batch_specs_c4()
    insts, keep = [], []
    alpha_solves_unknowns = 0
    for s in specs:
        grid = bi.Grid(s["dim"], tuple(s["M"]), 1.0, 0.1, s["nt"])
        rng = np.random.default_rng(s["seed"])
        modes = [(1,), (2,), (3,)] if grid.dim == 1 else [(1, 1), (2, 1), (1, 2)]
        z0 = bi.sine_field(grid, modes, rng.uniform(0.3, 1.0, 3))
        gd, delta = bi.add_noise_gaussian(grid, bi.forward_discrete(grid, z0), s["rel_noise"], rng)
        g = torch.as_tensor(gd.ravel(), dtype=torch.float64, device=device)
        y0 = torch.empty(grid.Nx, dtype=torch.float64, device=device)
        keep.append((g, y0, grid, gd, delta))
        insts.append(dict(dim=grid.dim, m=grid.M, L=1.0, T=0.1, nt=grid.nt, form=Q.FORM_PQ, delta=delta, g=g, y0=y0))
        alpha_solves_unknowns += grid.unknowns
    out = {"workload": "c4_batch_512_uneven_x16_alpha", "instances": len(specs), "n_alpha": 16}
    for name, prec in (("fp32_scan", Q.FP32_REFINE), ("fp64_scan", Q.FP64)):
        with Q.Sweep(insts, n_alpha=16, log10_lo=-1.5, log10_hi=1.5, tau_dp=1.1, precision=prec) as sw:
            cfg = sw.autotune(repeats=2, stream=stream)
            steps = max(3, args.steps // 4)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                sw.run(stream)
                e0.record(stream)
                for _ in range(steps):
                    sw.run(stream)
                e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            al, disc, err, pick = sw.read(stream)
            out[name] = {"ms_per_run": ms, "alpha_solves_per_s": len(specs) * 16 / (ms / 1e3),
                         "all_at_once_unknowns_per_s": 16 * alpha_solves_unknowns / (ms / 1e3),
                         "config": {"modes_per_thread": cfg.modes_per_thread, "ctas_per_sm": cfg.ctas_per_sm,
                                    "grid": cfg.grid},
                         "graph_launches_per_run": 1, "kernel_launches_per_run": 1}
            if with_oracle:
                out[name].update(_c4_oracle_check(keep, al, disc, pick))
    out["fp32_scan"]["mode"] = "alpha scan in FP32, y0 at the pick summed in double-float"
    out["fp64_scan"]["mode"] = ("alpha scan and y0 at the pick summed in double-float on the FP32 pipes "
                                "(about 2^-46 per term), DSTs in FP64")
    return out


def _c4_oracle_check(keep, al, disc, pick, tau_dp=1.1, count=4):
    """Discrepancies (all alphas), pick and y^0 at the pick of the `count`
    smallest instances against the oracle's full FP64 solves."""
    import numpy as np
    import bhcp_inputs as bi
    import oracle as O
    order = sorted(range(len(keep)), key=lambda i: keep[i][2].unknowns)[:count]
    dmax, ymax, same = 0.0, 0.0, 0
    for i in order:
        _, y0, grid, gd, delta = keep[i]
        od, oy = [], []
        for a in al[i]:
            y = O.solve_spectral(grid, O.PQ, float(a), O.delta_rhs(grid, O.PQ, float(a), gd))
            od.append(bi.discrete_l2(y[-1] - gd, grid))
            oy.append(y[0])
        od = np.array(od)
        dmax = max(dmax, float(np.max(np.abs(np.asarray(disc[i]) / od - 1.0))))
        ok = np.nonzero(od <= tau_dp * delta)[0]
        opick = int(ok[np.argmax(np.asarray(al[i])[ok])]) if len(ok) else int(np.argmin(od))
        same += int(int(pick[i, 0]) == opick)
        ymax = max(ymax, O.rel_l2(y0.cpu().numpy(), oy[int(pick[i, 0])].ravel()))
    return {"disc_rel_err_vs_oracle": dmax, "y0_at_pick_rel_err_vs_oracle": ymax,
            "picks_equal_to_oracle": f"{same}/{len(order)}",
            "oracle_sample": f"the {len(order)} smallest instances, all 16 alphas"}


def c4_full_leg(args, device, stream, with_oracle=True):
    """Full solves (every level, FP64) of the 512 uneven instances of the sweep
    workload (1D n in {63..2047}, 2D {63,127,255}^2, nt in {32..512}), alpha =
    each instance's noise level: one persistent launch from a captured CUDA
    graph (qbvm_multi_run) against the same instances as 512 single-plan
    solves one after another; sampled small instances against the oracle."""
    import numpy as np
    import torch
    import bhcp_inputs as bi
    import paper_2107_06381_gb300 as Q
    specs = bi.batch_specs_c4()
    insts, plans, meta = [], [], []
    for s_ in specs:
        grid = bi.Grid(s_["dim"], tuple(s_["M"]), 1.0, 0.1, s_["nt"])
        rng = np.random.default_rng(s_["seed"])
        modes = [(1,), (2,), (3,)] if grid.dim == 1 else [(1, 1), (2, 1), (1, 2)]
        z0 = bi.sine_field(grid, modes, rng.uniform(0.3, 1.0, 3))
        gd, delta = bi.add_noise_gaussian(grid, bi.forward_discrete(grid, z0), s_["rel_noise"], rng)
        g = torch.as_tensor(gd.ravel(), dtype=torch.float64, device=device)
        y = torch.empty(grid.unknowns, dtype=torch.float64, device=device)
        insts.append(dict(dim=grid.dim, m=grid.M, L=1.0, T=0.1, nt=grid.nt, form=Q.FORM_PQ, alpha=delta,
                          rhs_kind=Q.RHS_DELTA, g_or_F=g, y=y))
        plans.append((Q.Plan(grid.dim, grid.M, 1.0, 0.1, grid.nt, Q.FORM_PQ, delta, 0.0, Q.FP64, Q.RHS_DELTA), g, y))
        meta.append((grid, delta, gd))
    unknowns = sum(g.unknowns for g, _, _ in meta)
    out = {"workload": "c4_full_solves_512_uneven", "instances": len(specs), "unknowns_per_run": unknowns,
           "output": "every level of every instance (FP64)"}
    steps = max(3, args.steps // 5)
    with Q.Multi(insts) as mp:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            mp.run(stream)
            e0.record(stream)
            for _ in range(steps):
                mp.run(stream)
            e1.record(stream)
        torch.cuda.synchronize()
        mp.check(stream)
        ms = e0.elapsed_time(e1) / steps
        info = mp.info
        ys = [y.clone() for _, _, y in plans] if with_oracle else None
        with torch.cuda.stream(stream):
            for pl, g, y in plans:
                pl.solve(g, y, stream=stream)
            e0.record(stream)
            for _ in range(steps):
                for pl, g, y in plans:
                    pl.solve(g, y, stream=stream)
            e1.record(stream)
        torch.cuda.synchronize()
        ms_single = e0.elapsed_time(e1) / steps
        out.update({"ms_per_run": ms, "value": unknowns / (ms / 1e3), "unit": UNIT,
                    "solves_per_s": len(specs) / (ms / 1e3), "kernel_launches_per_run": 1,
                    "graph_launches_per_run": 1, "work_items": info["work_items"], "grid": info["grid"],
                    "single_plans_ms_per_run": ms_single,
                    "single_plans_kernel_launches_per_run": sum(p.info.kernels_per_solve for p, _, _ in plans)})
        if with_oracle:
            import oracle as O
            small = sorted(range(len(specs)), key=lambda i: meta[i][0].unknowns)[:4]
            errs, diffs = [], []
            for i in small:
                grid, delta, gd = meta[i]
                want = O.solve_spectral(grid, O.PQ, delta, O.delta_rhs(grid, O.PQ, delta, gd))
                errs.append(O.rel_l2(ys[i].cpu().numpy(), want))
            for i in range(0, len(specs), 64):
                a, b = ys[i], plans[i][2]
                diffs.append(float((a - b).norm() / b.norm()))
            out["rel_err_vs_oracle"] = max(errs)
            out["rel_err_sample"] = "the four smallest instances"
            out["rel_diff_vs_single_plans"] = max(diffs)
    for pl, _, _ in plans:
        pl.close()
    return out


def c1_batched_leg(args, device, stream, flush, count=10_000, with_oracle=True):
    """The 1D problem (63 interior points x 64 levels, T = 0.1, z0 = sin(pi x) +
    0.5 sin(3 pi x), multiplicative uniform noise eps = 1e-3) as a batch of
    `count` instances with their own noise draw and alpha = their own delta
    (PinT-QBVM, Section 5), full y of every instance, one qbvm_solve_batched
    call per batch: FP64 (3 kernel launches for the whole batch) and FP32
    transforms + double-float refinement (one launch: a CTA per instance runs
    the whole refinement in shared memory; one synchronisation per batch),
    each with its error against the FP64 oracle on sampled instances."""
    import numpy as np
    import torch
    import bhcp_inputs as bi
    import paper_2107_06381_gb300 as Q
    base = bi.make_c1()
    grid = base.grid
    rng = np.random.default_rng(101)
    g = base.g[None, :] * (1.0 + 1e-3 * rng.uniform(-1.0, 1.0, size=(count, grid.Nx)))
    alphas = np.sqrt(grid.h[0]) * np.linalg.norm(g - base.g[None, :], axis=1)      # grid-weighted delta
    gd = torch.as_tensor(g.ravel(), dtype=torch.float64, device=device)
    y = torch.empty(count * grid.unknowns, dtype=torch.float64, device=device)
    out = {"workload": f"c1_1d_63x64_batch{count}_delta_rhs", "instances": count,
           "unknowns_per_batch": count * grid.unknowns, "l2": "flushed between batches; output 322 MB"}
    sample = (0, 1, count // 2, count - 1)
    for name, prec in (("fp64", Q.FP64), ("fp32_refine", Q.FP32_REFINE)):
        with Q.Batch(1, grid.M, grid.L, grid.T, grid.nt, Q.FORM_PQ, alphas=list(alphas), rhs_kind=Q.RHS_DELTA,
                     precision=prec) as bt:
            steps = max(3, args.steps // 2)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            with torch.cuda.stream(stream):
                for _ in range(3):
                    bt.solve(gd, y, stream=stream)
                for i in range(steps):
                    evs[i][0].record(stream)
                    bt.solve(gd, y, stream=stream)
                    evs[i][1].record(stream)
                    flush.zero_()
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in evs) / steps
            leg = {"ms_per_batch": ms, "value": count * grid.unknowns / (ms / 1e3), "unit": UNIT,
                   "solves_per_s": count / (ms / 1e3)}
            if prec == Q.FP64:
                leg["kernel_launches_per_batch"] = 3
            else:
                it, rel = bt.refine_info
                leg.update({"refine_steps": it, "max_rel_residual": rel,
                            "dtype": "f32 transforms + double-float residual/update",
                            "one_launch": bt.refine_fused,
                            "kernel_launches_per_batch": 1 if bt.refine_fused else None})
            if with_oracle:
                import oracle as O
                errs = []
                for b in sample:
                    want = O.solve_spectral(grid, O.PQ, float(alphas[b]),
                                            O.delta_rhs(grid, O.PQ, float(alphas[b]), g[b]))
                    got = y[b * grid.unknowns:(b + 1) * grid.unknowns].cpu().numpy()
                    errs.append(O.rel_l2(got, want))
                leg["rel_err_vs_oracle"] = max(errs)
                leg["rel_err_sample"] = f"instances {list(sample)}"
            out[name] = leg
    # headline keys of the row: the FP64 batch (as before)
    out.update({k: out["fp64"][k] for k in ("ms_per_batch", "value", "unit", "solves_per_s")})
    out["kernel_launches_per_batch"] = 3
    out["fp32_refine_over_fp64_solves_per_s"] = out["fp32_refine"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    return out


def batched_2d_leg(args, device, stream, flush, count=64, with_oracle=True):
    """A batch of `count` 2D instances of the learned-alpha shape (127^2
    interior points x 128 levels, T = 0.1, 16 decaying sine modes, relative
    noise log-uniform in [1e-4, 1e-2]), alpha = each instance's delta, full y:
    the FP64 batch against the FP32 + double-float refinement batch, each with
    its error against the FP64 oracle on two sampled instances."""
    import numpy as np
    import torch
    import bhcp_inputs as bi
    import paper_2107_06381_gb300 as Q
    grid, z0, gd, delta = bi.alpha_training_batch(count, 77, M=128, nt=128, T=0.1)
    g = torch.as_tensor(gd.reshape(count, -1), dtype=torch.float64, device=device).contiguous()
    y = torch.empty(count * grid.unknowns, dtype=torch.float64, device=device)
    out = {"workload": f"batch{count}_2d_127sq_x128_delta_rhs", "instances": count,
           "unknowns_per_batch": count * grid.unknowns, "l2": "flushed between batches; output 1.06 GB"}
    for name, prec in (("fp64", Q.FP64), ("fp32_refine", Q.FP32_REFINE)):
        with Q.Batch(2, grid.M, grid.L, grid.T, grid.nt, Q.FORM_PQ, alphas=list(delta), rhs_kind=Q.RHS_DELTA,
                     precision=prec) as bt:
            steps = max(3, args.steps // 4)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            with torch.cuda.stream(stream):
                bt.solve(g, y, stream=stream)
                for i in range(steps):
                    evs[i][0].record(stream)
                    bt.solve(g, y, stream=stream)
                    evs[i][1].record(stream)
                    flush.zero_()
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in evs) / steps
            leg = {"ms_per_batch": ms, "value": count * grid.unknowns / (ms / 1e3), "unit": UNIT,
                   "solves_per_s": count / (ms / 1e3)}
            if prec == Q.FP32_REFINE:
                it, rel = bt.refine_info
                leg.update({"refine_steps": it, "max_rel_residual": rel})
            if with_oracle:
                import oracle as O
                errs = []
                for b in (0, count - 1):
                    a = float(delta[b])
                    want = O.solve_spectral(grid, O.PQ, a, O.rhs_block0(O.PQ, a, grid.tau, gd[b]), levels=[0, 127])
                    got = y[b * grid.unknowns:(b + 1) * grid.unknowns].view(grid.full_shape)[[0, 127]].cpu().numpy()
                    errs.append(O.rel_l2(got, want))
                leg["rel_err_vs_oracle_sampled_levels"] = max(errs)
            out[name] = leg
    out["fp32_refine_over_fp64_solves_per_s"] = out["fp32_refine"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    return out


# ------------------------------------------------------------ reference arm

def reference_arm(args):
    """The CPU FP64 oracle as it stands, on this host's cores; one step = the
    same two solves as the GPU arm's step (PinT-QBVM and PinT-MQBVM)."""
    import oracle as O
    prob = workload()
    grid = prob.grid
    forms = [O.PQ, O.PM]
    for i in range(args.warmup):
        cpu_oracle_leg(prob, forms, 2)
    t0 = time.perf_counter()
    _, times, _ = cpu_oracle_leg(prob, forms, 2 * args.steps)
    total = time.perf_counter() - t0
    value = grid.unknowns * len(forms) * args.steps / total
    cores = _cores_used()
    sample = ("two full 255^2 x 256 solves per step (PinT-QBVM and PinT-MQBVM) by the FP64 "
              "sine-basis oracle")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": headline_config(args, grid, len(forms), f"replicas{args.gpus}"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def learned_alpha_leg(n_train=8192, n_eval=1024, seed=5, with_oracle=True):
    """Learned alpha, bounded for the default run: train on n_train method-
    labelled 2D 127^2 x 128 instances (labels from the batched 32-alpha sweep,
    the alpha with the smallest ||y^0 - z0||), evaluate n_eval held-out ones.

    Three ways to pick alpha, each ending in y^0 of every held-out instance
    from the same FP64 sweep kernel (one persistent launch per batch):
      learned     features (sine spectrum) + MLP + one y^0 solve at its alpha;
      a_priori    one y^0 solve at alpha = delta (Section 5), the plain path;
      fp64_scan   32 alphas per instance; best-of-scan and the discrepancy
                  principle's pick (what the plain path needs to match the
                  learned accuracy without a network).
    Instances/s are wall-clock from g_delta resident on the device to y^0 and
    the errors read back, plan set-up included.  Mean e_h is the grid-weighted
    ||y^0 - z0|| (as the sweep reports it); `rel_err_vs_oracle` compares y^0 of sampled
    instances with the FP64 oracle's solve at the same alpha."""
    import numpy as np
    import torch
    import bhcp_inputs as bi
    import paper_2107_06381_gb300 as Q
    from paper_2107_06381_gb300 import learned_alpha as LA
    t0 = time.perf_counter()
    data = LA.make_dataset(n_train, seed=seed, chunk=4096)
    t_label = time.perf_counter() - t0
    mlp, hist = LA.train(data, epochs=12, batch=1024, lr=2e-3, seed=seed)
    grid, z0, gd, delta = bi.alpha_training_batch(n_eval, (seed + 1) * 1000003, M=128, nt=128, T=0.1)
    g_dev = torch.as_tensor(gd.reshape(n_eval, -1), dtype=torch.float64).cuda()
    z_dev = torch.as_tensor(z0.reshape(n_eval, -1), dtype=torch.float64).cuda()
    y0s = {k: torch.empty((n_eval, grid.Nx), dtype=torch.float64, device="cuda")
           for k in ("learned", "a_priori")}
    fplan = Q.Features(128, 0.1, 128, n_eval)
    feats = torch.empty((n_eval, LA.IN_DIM), dtype=torch.float32, device="cuda")
    tpred = torch.empty(n_eval, dtype=torch.float32, device="cuda")

    def sweep(n_alpha, lo, hi, base, y0):
        insts = [dict(dim=2, m=grid.M, L=1.0, T=0.1, nt=128, form=Q.FORM_PQ, delta=float(delta[b]),
                      alpha_base=0.0 if base is None else float(base[b]), g=g_dev[b], z0=z_dev[b],
                      y0=None if y0 is None else y0[b]) for b in range(n_eval)]
        with Q.Sweep(insts, n_alpha=n_alpha, log10_lo=lo, log10_hi=hi, tau_dp=1.1, precision=Q.FP64) as sw:
            sw.run()
            return sw.read()

    out = {"workload": "learned_alpha_2d_127sq_x128", "train_instances": n_train, "eval_instances": n_eval,
           "labels_from": "batched sweep, 32 alphas in [alpha_rule/100, 100 alpha_rule], min ||y0 - z0||",
           "label_and_feature_seconds": round(t_label, 2),
           "train_loss_first_last": [round(hist[0][1], 4), round(hist[-1][1], 4)], "data": "synthetic"}
    res = {}
    for rep in range(2):                       # the first pass warms up every plan path
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fplan.run(g_dev, delta, feats)
        mlp.forward(feats, tpred)
        t_l = tpred.cpu().numpy().astype(np.float64)
        al_l, _, err_l, _ = sweep(1, 0.0, 0.0, delta * 10.0 ** t_l, y0s["learned"])
        s_learned = time.perf_counter() - t0
        t0 = time.perf_counter()
        al_r, _, err_r, _ = sweep(1, 0.0, 0.0, None, y0s["a_priori"])
        s_rule = time.perf_counter() - t0
        t0 = time.perf_counter()
        al_s, disc_s, err_s, pick_s = sweep(LA.N_ALPHA, LA.LOG_LO, LA.LOG_HI, None, None)
        s_scan = time.perf_counter() - t0
        res = {"learned": (err_l[:, 0], s_learned), "a_priori": (err_r[:, 0], s_rule),
               "fp64_scan_best": (err_s.min(axis=1), s_scan),
               "fp64_scan_discrepancy": (err_s[np.arange(n_eval), pick_s[:, 0]], s_scan)}
    for k, (err, secs) in res.items():
        out[k] = {"mean_e_h": float(np.mean(err)), "instances_per_s": n_eval / secs}
    out["learned_better_than_rule_fraction"] = float(np.mean(res["learned"][0] < res["a_priori"][0]))
    out["learned_alpha_over_rule_log10_mean"] = float(np.mean(t_l))
    if with_oracle:
        import oracle as O
        errs = []
        for name, al in (("learned", al_l), ("a_priori", al_r)):
            for b in (0, n_eval - 1):
                a = float(al[b, 0])
                want = O.solve_spectral(grid, O.PQ, a, O.rhs_block0(O.PQ, a, grid.tau, gd[b]), levels=[0])
                got = y0s[name][b].cpu().numpy().reshape(want.shape)
                errs.append(O.rel_l2(got, want))
        out["rel_err_vs_oracle"] = max(errs)
        out["rel_err_sample"] = "y0 of the first and last held-out instance, learned and a-priori alpha"
    fplan.close()
    mlp.close()
    return out


def c5_leg(n_train=200_000, n_eval=4096, seed=5):
    """Learned alpha at its full size: 2D 127^2 x 128 instances (16 decaying sine
    modes, relative noise log-uniform in [1e-4, 1e-2]); labels from the batched
    32-alpha sweep (the alpha with the smallest ||y^0 - z0||), features and the
    MLP on the GPU; evaluation on held-out instances against the a-priori rule
    alpha = delta, the discrepancy principle and the scan's best."""
    import numpy as np
    import torch
    import paper_2107_06381_gb300 as Q
    from paper_2107_06381_gb300 import learned_alpha as LA
    Q.build_library()
    Q.load_library()
    t0 = time.perf_counter()
    data = LA.make_dataset(n_train, seed=seed, chunk=4096)
    t_label = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mlp, hist = LA.train(data, epochs=12, batch=1024, lr=2e-3, seed=seed)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    ev = LA.evaluate(mlp, n_eval, seed=seed + 1, chunk=4096)
    mlp.close()
    return {"workload": "c5_learned_alpha_2d_127sq_x128", "train_instances": n_train, "eval_instances": n_eval,
            "labels_from": "batched sweep, 32 alphas in [alpha_rule/100, 100 alpha_rule], min ||y0 - z0||",
            "label_and_feature_seconds": round(t_label, 2), "train_seconds": round(t_train, 2),
            "train_loss_first_last": [round(hist[0][1], 4), round(hist[-1][1], 4)],
            "mean_e_h": {"learned": float(ev["learned"].mean()), "a_priori_rule": float(ev["rule"].mean()),
                         "discrepancy_principle": float(ev["morozov"].mean()), "best_of_scan": float(ev["best"].mean())},
            "learned_better_than_rule_fraction": float(np.mean(ev["learned"] < ev["rule"])),
            "one_alpha_solves_per_s": float(ev["one_alpha_solves_per_s"]),
            "scan_alpha_solves_per_s": float(ev["scan_solves_per_s"]),
            "scan_instances_per_s": float(ev["scan_instances_per_s"]),
            "data": "synthetic"}


def run_legs(args, device, stream, flush, with_oracle, only=None):
    """The secondary workloads (3D, the sweeps, the batches, learned alpha),
    all of them or the one named."""
    legs = {
        "c3_3d": lambda: c3_leg(args, device, stream, flush, with_oracle),
        "c4_sweep": lambda: c4_leg(args, device, stream, with_oracle=with_oracle),
        "c4_full_multi": lambda: c4_full_leg(args, device, stream, with_oracle=with_oracle),
        "c1_batched": lambda: c1_batched_leg(args, device, stream, flush, with_oracle=with_oracle),
        "batched_2d": lambda: batched_2d_leg(args, device, stream, flush, with_oracle=with_oracle),
        "learned_alpha": lambda: learned_alpha_leg(with_oracle=with_oracle),
    }
    return {k: f() for k, f in legs.items() if only is None or k == only}


def main():
    args = parse()
    if args.leg:
        import torch
        import paper_2107_06381_gb300 as Q
        device = torch.device("cuda", 0)
        torch.cuda.set_device(device)
        Q.build_library()
        Q.load_library()
        stream = torch.cuda.Stream(device)
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)      # 256 MB > L2
        print(json.dumps(run_legs(args, device, stream, flush, not args.no_cpu_baseline, only=args.leg)), flush=True)
        return 0
    if args.c5:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(c5_leg()), flush=True)
        return 0
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(reference_arm(args)), flush=True)
        return 0
    import torch
    device = torch.device("cuda", local_rank)
    torch.cuda.set_device(device)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=device)
    out = our_arm(args, rank, world, device)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
