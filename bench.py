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
# FP64 ALU peak derived from the part's unit counts and clock: 152 SMs x 2 FP64
# operations (DADD, DMUL or DFMA) per clock x 2.07 GHz.
FP64_PEAK_TOPS = 152 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + write) per launch from one ncu capture of the current
# kernels on this workload (profiles/); None once a kernel changes.
PROFILED_TRAFFIC = {"dst_x": 133.416704e6 + 84.831488e6, "dst_y": 133.236992e6 + 77.190912e6,
                    "time_solve": 266.473728e6 + 89.289984e6}


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

    # ---- timed region
    for plan in plans:
        plan.profile(True)
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
    kstats = {}
    for plan in plans:
        for name, (launches, ms) in plan.profile_read().items():
            a, b = kstats.get(name, (0, 0.0))
            kstats[name] = (a + launches, b + ms)
        plan.profile(False)
    launches_per_solve = plans[0].info.kernels_per_solve
    unknowns_step = grid.unknowns * len(forms)
    value = world * unknowns_step * args.steps / (total_ms / 1e3) if total_ms > 0 else 0.0

    # ---- roofline of the dominant kernel
    hbm_peak, hbm_src = _peaks()
    if not kstats:
        kstats = {"none": (1, 1e-9)}
    dom = max(kstats.items(), key=lambda kv: kv[1][1])
    dname, (dl, dms) = dom
    byts, ops = kernel_model(dname, grid, args.rhs)
    avg_s = dms / dl / 1e3
    roof = None
    if byts is not None:
        t_hbm = byts / (hbm_peak * 1e9)
        t_alu = ops / (FP64_PEAK_TOPS * 1e12)
        traffic = PROFILED_TRAFFIC.get(dname)
        if t_alu > t_hbm:
            ach = ops / avg_s / 1e12
            roof = {"bound": "alu", "kernel": dname, "achieved": round(ach, 4), "peak": round(FP64_PEAK_TOPS, 4),
                    "unit": "T FP64-op/s (DADD/DMUL/DFMA = 1 op)", "frac": round(ach / FP64_PEAK_TOPS, 4),
                    "traffic": traffic,
                    "peak_source": "derived: 152 SMs x 2 FP64 ops/clk x 2.07 GHz",
                    "hbm_achieved_gbs": round(byts / avg_s / 1e9, 1),
                    "hbm_frac": round(byts / avg_s / 1e9 / hbm_peak, 4), "hbm_peak_source": hbm_src}
        else:
            ach = byts / avg_s / 1e9
            roof = {"bound": "hbm", "kernel": dname, "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(ach / hbm_peak, 4), "traffic": traffic, "peak_source": hbm_src}
        # the other two HBM figures: DRAM bytes ncu measured for this kernel over its
        # event-timed duration, and the whole solve's algorithmic bytes (F in + y
        # out, or g in + y out) at the measured unknowns/s -- both over the copy peak
        bpu = 16 if args.rhs == "general" else 8
        roof["dram_gbs_ncu"] = round(traffic / avg_s / 1e9, 1) if traffic else None
        roof["dram_frac_ncu"] = round(traffic / avg_s / 1e9 / hbm_peak, 4) if traffic else None
        roof["solve_algorithmic_gbs"] = round(bpu * value / 1e9, 1)
        roof["solve_algorithmic_frac"] = round(bpu * value / 1e9 / hbm_peak, 4)
    kernels = {k: {"launches": v[0], "avg_ms": round(v[1] / v[0], 4), "share": round(v[1] / sum(x[1] for x in kstats.values()), 4)}
               for k, v in sorted(kstats.items(), key=lambda kv: -kv[1][1])}

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
        for plan in rplans:
            plan.profile(True)
        revs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                revs[i][0].record(stream)
                rstep()
                revs[i][1].record(stream)
                flush.zero_()
        torch.cuda.synchronize(device)
        r_ms = sum(a.elapsed_time(b) for a, b in revs)
        rk = {}
        for plan in rplans:
            for name, (launches, ms) in plan.profile_read().items():
                a, b = rk.get(name, (0, 0.0))
                rk[name] = (a + launches, b + ms)
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
        extra["c3_3d"] = c3_leg(args, device, stream, flush, rank == 0 and world == 1 and not args.no_cpu_baseline)
        extra["c4_sweep"] = c4_leg(args, device, stream)
        extra["c1_batched"] = c1_batched_leg(args, device, stream, flush)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"c2_2d_255sq_x256_{args.rhs}_rhs", "dim": 2, "interior": [255, 255], "nt": 256,
                   "T": grid.T, "forms": ["pint-qbvm", "pint-mqbvm"], "rhs": args.rhs,
                   "unknowns_per_solve": grid.unknowns, "solves_per_step": len(forms),
                   "l2": "flushed between steps (256 MB write outside the timed events); inputs 133 MB/solve",
                   "parallelism": f"replicas{world}"},
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


def c4_leg(args, device, stream):
    """512 uneven instances (1D n in {63..2047}, 2D {63,127,255}^2, nt in {32..512},
    relative noise log-uniform in [1e-4, 1e-2]) x 16 alphas, one persistent
    launch per run from a captured CUDA graph, launch shape autotuned."""
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
        keep.append((g, y0))
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
    return out


def c1_batched_leg(args, device, stream, flush, count=10_000):
    """The 1D problem (63 interior points x 64 levels, T = 0.1, z0 = sin(pi x) +
    0.5 sin(3 pi x), multiplicative uniform noise eps = 1e-3) as a batch of
    `count` instances with their own noise draw and alpha = their own delta
    (PinT-QBVM, Section 5), full y of every instance: one qbvm_solve_batched
    call = 3 kernel launches for the whole batch."""
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
           "unknowns_per_batch": count * grid.unknowns}
    with Q.Batch(1, grid.M, grid.L, grid.T, grid.nt, Q.FORM_PQ, alphas=list(alphas), rhs_kind=Q.RHS_DELTA) as bt:
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
        # two instances against single-instance plans (the same kernels, one instance each)
        diffs = []
        for b in (0, count - 1):
            with Q.Plan(1, grid.M, grid.L, grid.T, grid.nt, Q.FORM_PQ, float(alphas[b]), 0.0, Q.FP64,
                        Q.RHS_DELTA) as plan:
                one = torch.empty(grid.unknowns, dtype=torch.float64, device=device)
                plan.solve(gd[b * grid.Nx:(b + 1) * grid.Nx].contiguous(), one)
                torch.cuda.synchronize()
                mine = y[b * grid.unknowns:(b + 1) * grid.unknowns]
                diffs.append(float((mine - one).norm() / one.norm()))
    out.update({"ms_per_batch": ms, "value": count * grid.unknowns / (ms / 1e3), "unit": UNIT,
                "solves_per_s": count / (ms / 1e3), "kernel_launches_per_batch": 3,
                "rel_diff_vs_single_instance_plans": max(diffs),
                "l2": "flushed between batches; output 322 MB"})
    return out


# ------------------------------------------------------------ reference arm

def reference_arm(args):
    """The CPU FP64 oracle as it stands, on this host's cores; one step = one
    formulation (alternating) of the same workload."""
    import oracle as O
    prob = workload()
    grid = prob.grid
    forms = [O.PQ, O.PM]
    for i in range(args.warmup):
        cpu_oracle_leg(prob, [forms[i % 2]], 1)
    t0 = time.perf_counter()
    _, times, _ = cpu_oracle_leg(prob, forms, args.steps)
    total = time.perf_counter() - t0
    value = grid.unknowns * args.steps / total
    cores = _cores_used()
    sample = ("one full 255^2 x 256 solve per step (PinT-QBVM and PinT-MQBVM alternating) by the FP64 "
              "sine-basis oracle")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"c2_2d_255sq_x256_{args.rhs}_rhs", "dim": 2, "interior": [255, 255], "nt": 256,
                       "parallelism": "cpu"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


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


def main():
    args = parse()
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
