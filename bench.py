"""Benchmark of the tau-preconditioned Krylov time stepping on one GB300.

Workload (one bench "step"): the 1D variable-coefficient FDE with n = 65535,
alpha in {1.2, 1.5, 1.8}, d+ = 1 + x^2, d- = 1 + (1-x)^2, 20 implicit-Euler
steps with dt = 1/512 from u0 = x^2(1-x)^2 + seeded noise, GMRES(30) with the
unshifted tau preconditioner, true relres 1e-8: 60 solves, the three alphas
batched in one persistent launch per time step.  Both precision paths are
timed (plain FP64; FP32 inner GMRES with FP64 refinement) and the faster one
that reaches relres 1e-8 on every solve is the headline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own copy of the workload on its GPU (the
solves are independent; no collective on the data path): weak scaling.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT = 65535
ALPHAS = (1.2, 1.5, 1.8)
TIME_STEPS = 20
RESTART = 30
TOL = 1e-8
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2
# dram__bytes_read.sum + dram__bytes_write.sum of one FP64 engine launch of this
# workload (balanced teams), from the ncu capture summarised under profiles/
F64_LAUNCH_DRAM_BYTES = 303.106304e6 + 804.658432e6
# FP64 ALU peak: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (the nominal 1.25 TFLOP/s)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP64_PEAK_SOURCE = "derived: 152 SM x 2 DFMA/clk x 2 x 2.07 GHz"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--precisions", default="f64,f32_ir")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--inner-tol", type=float, default=1e-3)
    ap.add_argument("--graph", type=int, default=1, help="1: replay the time-step loop as a CUDA graph")
    ap.add_argument("--batch", type=int, default=1, help="1: also time the 256-instance batched workload")
    ap.add_argument("--two-d", type=int, default=1, help="1: also time the two 2D workloads")
    ap.add_argument("--only", default="", choices=["", "2d", "batch"],
                    help="time only this section and print its results (for profiling one kernel)")
    ap.add_argument("--autotune", type=int, default=1,
                    help="1: pick each plan's transform schedule with fde_autotune before timing")
    ap.add_argument("--variants", type=int, default=1,
                    help="1: also time the preconditioner variants in FP64: the shift c0/mean(D) beside D, "
                         "and P_F-tilde (D folded into the symbol)")
    ap.add_argument("--balance", type=int, default=1,
                    help="1: team sizes follow the previous time step's iteration counts")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
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
        sm, mx, reasons = [], None, set()
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for name, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def algorithmic_per_iteration(n: int, elem: int):
    """Per Arnoldi iteration of right-preconditioned GMRES(30) on one 1D line:
    40 vector passes of n elements (tau solve 3, matvec 4, classical
    Gram-Schmidt with one reorthogonalisation about 2 (j+1) + 4 with j ~ m/2)
    and 12.5 L log2 L flops (five real-packed FFTs of n+1 points), L = 2(n+1)."""
    L = 2 * (n + 1)
    return 40 * elem * n, 12.5 * L * math.log2(L)


def run_ours(args, rank, world, device):
    import numpy as np
    import torch

    import paper_1912_13304_gb300 as fde
    import workloads
    from paper_1912_13304_gb300 import build as fbuild

    fbuild.build()
    fde.lib()
    n = args.n
    ws = workloads.var_1d_time_stepping(n=n, alphas=ALPHAS, steps=TIME_STEPS)
    u0_host = [torch.tensor(w["u0"], dtype=torch.float64).pin_memory() for w in ws]
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    fp64_peak_tflops = FP64_PEAK_TFLOPS

    results = {}
    from paper_1912_13304_gb300.solver import TimeStepper

    runs = [(p, "") for p in args.precisions.split(",") if p]
    if args.variants:
        runs += [("f64", "shift"), ("f64", "ftilde")]
    for prec, variant in runs:
        key = prec + ("+" + variant if variant else "")
        plans = [fde.Plan.from_workload(w, precision=prec, shift=variant == "shift",
                                        order="tau_df" if variant == "ftilde" else None, device=device)
                 for w in ws]
        schedule = [p.autotune() for p in plans][0] if args.autotune else (0, 0)
        u = [torch.empty(n, dtype=torch.float64, device=device) for _ in ws]
        kw = dict(tol=TOL, max_iters=20000, inner_tol=args.inner_tol, max_outer=200, balance=bool(args.balance))
        u0_dev = [x.to(device) for x in u0_host]

        def reset():
            for k in range(len(ws)):
                u[k].copy_(u0_dev[k])
            flush.fill_(1.0)

        # eager warm-up (also the launch-duration pass below), then the loop of
        # TIME_STEPS steps captured once as a CUDA graph
        eager = TimeStepper(plans, u, TIME_STEPS, graph=False, **kw)
        for _ in range(args.warmup):
            reset()
            eager.run()
        torch.cuda.synchronize()
        stepper = TimeStepper(plans, u, TIME_STEPS, graph=bool(args.graph), **kw)
        for _ in range(args.warmup):
            reset()
            stepper.run()
        torch.cuda.synchronize()
        # timed region: K bench steps (graph replays), L2 flushed before each, device events
        step_ms = []
        with ClockSampler(torch.cuda.current_device()) as clk:
            for _ in range(args.steps):
                reset()
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                if world > 1:
                    torch.distributed.barrier()
                torch.cuda.synchronize()
                s0.record()
                stepper.run()
                s1.record()
                torch.cuda.synchronize()
                step_ms.append(s0.elapsed_time(s1))
        infos = [i for step in stepper.infos() for i in step]
        its = sum(i["iterations"] for i in infos)
        worst = max(i["relres"] for i in infos)
        ok = all(i["status"] == fde.OK and i["relres"] <= TOL for i in infos)
        # duration of each solve launch: the same steps as eager launches with events around each
        launch_ms = []
        for _ in range(args.steps):
            reset()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(TIME_STEPS)]
            eager.run_eager(ev)
            torch.cuda.synchronize()
            launch_ms += [a.elapsed_time(c) for a, c in ev]
        # end to end: inputs from pinned host memory, solution back to host, every step
        e2e_ms = []
        out_host = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in ws]
        for _ in range(max(1, args.steps)):
            flush.fill_(1.0)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            s0.record()
            for k in range(len(ws)):
                u[k].copy_(u0_host[k], non_blocking=True)
            stepper.run()
            for k in range(len(ws)):
                out_host[k].copy_(u[k], non_blocking=True)
            s1.record()
            torch.cuda.synchronize()
            e2e_ms.append(s0.elapsed_time(s1))
        elem = 8 if prec == "f64" else 4
        bpi, fpi = algorithmic_per_iteration(n, elem)
        per_launch_its = its / (TIME_STEPS)
        avg_launch = sum(launch_ms) / len(launch_ms)
        if prec == "f64":
            achieved = per_launch_its * fpi / (avg_launch * 1e-3) / 1e12
            # DRAM read + write of one balanced FP64 launch (ncu; profiles/fde_engine_f64_n65535_3alpha.md)
            roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                    "frac": achieved / fp64_peak_tflops, "traffic": F64_LAUNCH_DRAM_BYTES if args.balance else None,
                    "peak_source": FP64_PEAK_SOURCE}
        else:
            achieved = per_launch_its * bpi / (avg_launch * 1e-3) / 1e9
            roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "traffic": None, "peak_source": hbm_src}
        t_step = sum(step_ms) / len(step_ms)
        nsolves = TIME_STEPS * len(ws)
        results[key] = dict(
            ms_per_step=t_step, solves_per_s=nsolves / (t_step * 1e-3),
            unknown_iters_per_s=n * its / (t_step * 1e-3), iterations=its,
            outer=sum(i["outer"] for i in infos), worst_relres=worst, converged=ok,
            e2e_ms=sum(e2e_ms) / len(e2e_ms), roofline=roof, clocks=clk.summary(),
            launch_ms=avg_launch, step_ms=step_ms, schedule={"ctas": schedule[0], "log_p1": schedule[1]})
        for p in plans:
            p.close()
    return results


def shard_by_cost(costs, world: int) -> list[list[int]]:
    """Partition instance indices over `world` ranks by cost, longest first
    onto the least-loaded rank (ties: lower index, lower rank).  Each rank's
    list is in ascending index order; with one rank it is every index in order."""
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(world), key=lambda r: (load[r], r))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def batch_cost(n: int) -> float:
    """Relative cost of one constant-coefficient PCG solve of size n: the
    Case I shifted preconditioner keeps the iteration count flat in n, so the
    work per solve goes as the line transforms, L log2 L with L = 2(n+1)."""
    L = 2 * (n + 1)
    return L * math.log2(L)


BATCH_KS = range(8, 15)        # n = 2^k - 1 of the batched workload


def batch_job(local: dict, world: int, device) -> dict:
    """Whole-job figures of the sharded batch (every rank calls it; a
    collective when world > 1): the slowest rank's launch time, the worst
    relres and per-size iteration maximum, summed iterations, flops and
    unknown-iterations, and whether every rank converged.  `max_its_by_k`
    holds one entry per k of BATCH_KS (0 where a rank has no such size)."""
    if world == 1:
        return dict(local)
    import torch
    mx = torch.tensor([local["ms_per_launch"], local["worst_relres"]] + list(local["max_its_by_k"]),
                      dtype=torch.float64, device=device)
    sm = torch.tensor([local["iterations"], local["outer"], local["unknown_iters"], local["flops"],
                       0.0 if local["converged"] else 1.0], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(mx, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(sm, op=torch.distributed.ReduceOp.SUM)
    return {"ms_per_launch": float(mx[0]), "worst_relres": float(mx[1]),
            "max_its_by_k": [int(v) for v in mx[2:].tolist()], "iterations": int(sm[0]), "outer": int(sm[1]),
            "unknown_iters": float(sm[2]), "flops": float(sm[3]), "converged": float(sm[4]) == 0.0}


def run_batch(args, device, rank: int = 0, world: int = 1):
    """The batched workload: 256 independent 1D constant-coefficient solves
    (n = 2^k - 1, k ~ U{8..14}; alpha ~ U(1.1, 1.9); d, dt per instance; seed
    2), PCG with each instance's shifted tau preconditioner, relres 1e-8, all
    in one persistent launch (one-CTA teams taking instances from a queue,
    largest first).  Reported per precision path: solves/s and
    unknown-iterations/s.  Under torchrun the instances are sharded over the
    ranks by cost (no collective on the data path; the 256 solves are the
    fixed total, strong scaling) and the figures are whole-job ones."""
    import torch

    import paper_1912_13304_gb300 as fde
    import workloads
    ws_all = workloads.const_1d_batch()
    mine = shard_by_cost([batch_cost(w["n1"]) for w in ws_all], world)[rank]
    ws = [ws_all[i] for i in mine]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    out = {}
    # the workload's own preconditioner (Case I shift) and the default layout:
    # one-CTA teams hold whole lines where they fit
    for prec in [p for p in args.precisions.split(",") if p]:
        plans = [fde.Plan.from_workload(w, precision=prec, device=device) for w in ws]
        bs = [p.c0 * torch.tensor(w["b"], dtype=torch.float64, device=device) for p, w in zip(plans, ws)]
        xs = [torch.zeros_like(b) for b in bs]
        info = torch.zeros(len(ws) * fde.INFO_BYTES, dtype=torch.uint8, device=device)

        def once():
            for x in xs:
                x.zero_()
            fde.solve_batch(plans, bs, xs, tol=TOL, max_iters=2000, inner_tol=1e-4, max_outer=100,
                            info_dev=info, read_info=False)

        for _ in range(args.warmup):
            once()
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            for x in xs:
                x.zero_()
            flush.fill_(1.0)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            s0.record()
            fde.solve_batch(plans, bs, xs, tol=TOL, max_iters=2000, inner_tol=1e-4, max_outer=100,
                            info_dev=info, read_info=False)
            s1.record()
            torch.cuda.synchronize()
            ms.append(s0.elapsed_time(s1))
        infos = fde.decode_info(info.cpu().numpy().tobytes(), len(ws))
        max_its = {k: 0 for k in BATCH_KS}
        for w, i in zip(ws, infos):
            k = int(round(math.log2(w["n1"] + 1)))
            max_its[k] = max(max_its[k], i["iterations"])
        job = batch_job({"ms_per_launch": sum(ms) / len(ms),
                         "worst_relres": max((i["relres"] for i in infos), default=0.0),
                         "max_its_by_k": [max_its[k] for k in BATCH_KS],
                         "iterations": sum(i["iterations"] for i in infos),
                         "outer": sum(i["outer"] for i in infos),
                         "unknown_iters": float(sum(w["n1"] * i["iterations"] for w, i in zip(ws, infos))),
                         "flops": sum(i["iterations"] * FFTS_PER_ITERATION["pcg"] * fft_flops(2 * (w["n1"] + 1))
                                      for w, i in zip(ws, infos)),
                         "converged": all(i["status"] == fde.OK and i["relres"] <= TOL for i in infos)},
                        world, device)
        t = job["ms_per_launch"]
        out[prec] = {"ms_per_launch": t, "solves_per_s": len(ws_all) / (t * 1e-3),
                     "max_iterations_by_n": {str(2 ** k - 1): v for k, v in zip(BATCH_KS, job["max_its_by_k"])
                                             if v > 0},
                     "unknown_iters_per_s": job["unknown_iters"] / (t * 1e-3),
                     "iterations": job["iterations"],
                     "outer": job["outer"],
                     "worst_relres": job["worst_relres"],
                     "converged": job["converged"]}
        if prec == "f64":
            out[prec]["roofline"] = alu_roofline(job["flops"], t, FP64_PEAK_TFLOPS * world)
        for p in plans:
            p.close()
    return {"workload": "batch256-1d-const-n255..16383-pcg-shifted-tau", "instances": len(ws_all),
            "unknowns": sum(w["n1"] for w in ws_all), "paths": out,
            "sharding": "one launch" if world == 1 else f"cost-balanced over {world} ranks (strong scaling)"}


# Algorithmic vector passes per iteration of the 2D solves (each pass reads or
# writes N elements once): PCG with P_hat about 11, GMRES(20) with D_N about 34.
PASSES_2D = {"pcg": 11, "gmres": 34}

# Real-packed FFTs of one line per iteration: the tau solve's two sine
# transforms, plus the matvec's forward and one inverse transform (PCG,
# symmetric multiplier) or two inverse transforms (GMRES, D_+ T x and D_- T^T x).
FFTS_PER_ITERATION = {"pcg": 4, "gmres": 5}


def fft_flops(L: int) -> float:
    """Flops of one real-packed FFT of L real points (an L/2-point complex FFT
    plus the pair step), the 2.5 L log2 L of the split-radix count."""
    return 2.5 * L * math.log2(L)


def alu_roofline(flops: float, ms: float, peak_tflops: float) -> dict:
    achieved = flops / (ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": achieved / peak_tflops, "traffic": None, "peak_source": FP64_PEAK_SOURCE}


def run_2d(args, device):
    """The two 2D workloads, one solve each per bench step: 2047^2 constant
    coefficients (alpha 1.5, beta 1.7, PCG with P_hat, seed 1) and 4095^2
    variable coefficients (alpha 1.3, beta 1.8, one implicit-Euler step from
    u0 = sin(pi x) sin(pi y), GMRES(20) with the 2D tau(F) D_N).  Reported per
    precision path: solves/s, unknown-iterations/s and the algorithmic HBM
    bandwidth (vector passes x element bytes x N per iteration) against the
    measured copy peak."""
    import torch

    import paper_1912_13304_gb300 as fde
    import workloads
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    out = {}
    w5 = workloads.var_2d_time_stepping(steps=1)
    w5cn = dict(w5, time_scheme="cn")
    for name, w in (("2d-const-n2047-pcg-phat", workloads.const_2d()),
                    ("2d-var-n4095-gmres20-one-step", w5),
                    ("2d-var-n4095-gmres20-crank-nicolson-step", w5cn)):
        res = {}
        N = w["n1"] * w["n2"]
        for prec in [p for p in args.precisions.split(",") if p]:
            if w.get("time_scheme") == "cn":
                # the same plane with the Crank-Nicolson scheme: the timed step
                # includes the explicit half b = (2 c0 I - M) u0 (fde_step_rhs)
                plan = fde.Plan(2, w["n1"], w["alpha"], w["dt"], n2=w["n2"], beta=w["beta"], len1=w["length"],
                                len2=w["length"], scheme="cn", weights=w["scheme"], dp=w["dp"].reshape(-1),
                                dm=w["dm"].reshape(-1), ep=w["ep"].reshape(-1), em=w["em"].reshape(-1),
                                method="gmres", restart=w["restart"], precision=prec, device=device)
            else:
                plan = fde.Plan.from_workload(w, precision=prec, device=device)
            schedule = plan.autotune() if args.autotune else (0, 0)
            cn = w.get("time_scheme") == "cn"
            if w["rhs_scale"] == "unit":
                b = plan.c0 * torch.tensor(w["b"], dtype=torch.float64, device=device)
                x0 = torch.zeros_like(b)
            else:
                x0 = torch.tensor(w["u0"], dtype=torch.float64, device=device)
                b = plan.rhs(x0)
            x = torch.empty_like(b)
            info = torch.zeros(fde.INFO_BYTES, dtype=torch.uint8, device=device)
            kw = dict(tol=TOL, max_iters=5000, inner_tol=1e-4, max_outer=100, info_dev=info, read_info=False)

            def step():
                if cn:
                    plan.rhs(x0, b=b)
                fde.solve_batch([plan], [b], [x], **kw)

            for _ in range(args.warmup):
                x.copy_(x0)
                step()
            torch.cuda.synchronize()
            ms = []
            for _ in range(args.steps):
                x.copy_(x0)
                flush.fill_(1.0)
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                s0.record()
                step()
                s1.record()
                torch.cuda.synchronize()
                ms.append(s0.elapsed_time(s1))
            inf = fde.decode_info(info.cpu().numpy().tobytes(), 1)[0]
            t = sum(ms) / len(ms)
            elem = 8 if prec == "f64" else 4
            gbs = inf["iterations"] * PASSES_2D[w["method"]] * elem * N / (t * 1e-3) / 1e9
            res[prec] = {"ms_per_solve": t, "solves_per_s": 1e3 / t,
                         "unknown_iters_per_s": N * inf["iterations"] / (t * 1e-3),
                         "iterations": inf["iterations"], "outer": inf["outer"], "relres": inf["relres"],
                         "converged": inf["status"] == fde.OK and inf["relres"] <= TOL,
                         "schedule": {"ctas": schedule[0], "log_p1": schedule[1]},
                         "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                                      "frac": gbs / hbm_peak, "traffic": None}}
            if prec == "f64":
                # the FP64 transforms bound this path, as in 1D: its HBM figure stays beside
                n1, n2 = w["n1"], w["n2"]
                flops = inf["iterations"] * FFTS_PER_ITERATION[w["method"]] * (
                    n2 * fft_flops(2 * (n1 + 1)) + n1 * fft_flops(2 * (n2 + 1)))
                res[prec]["roofline_hbm"] = res[prec]["roofline"]
                res[prec]["roofline"] = alu_roofline(flops, t, FP64_PEAK_TFLOPS)
            plan.close()
            del x, b, x0
            torch.cuda.empty_cache()
        out[name] = {"unknowns": N, "paths": res}
    return out


def oracle_sample(n: int, cap: int = 4):
    """The oracle on the first implicit-Euler solve of the alpha = 1.8 line of
    size n (direct Toeplitz sums, library DST-I), capped at `cap` GMRES
    iterations: (seconds, iterations).  Module level, so spawned worker
    processes can run it."""
    import oracle
    import workloads
    w = workloads.var_1d_time_stepping(n=n, alphas=(1.8,))[0]
    h = 1.0 / (n + 1)
    prob = oracle.Problem1D(alpha=w["alpha"], n=n, c0=h ** w["alpha"] / w["dt"], dp=w["dp"], dm=w["dm"])
    P = oracle.Tau1D.for_problem(prob)
    b = prob.c0 * w["u0"]
    t0 = time.perf_counter()
    res = oracle.gmres(prob.matvec, b, Pinv=P.apply_inverse, x0=w["u0"], restart=RESTART, tol=TOL, maxiter=cap)
    return time.perf_counter() - t0, max(res.iterations, 1)


def cpu_baseline_sample(n: int, all_cores: bool = False):
    """The oracle as it stands on a bounded sample of the workload: the
    first implicit-Euler solve of the alpha = 1.8 line, n = 65535, with the
    oracle's direct (non-FFT) Toeplitz sums and library DST-I, capped at 4
    GMRES iterations; scaled to solves/s with the oracle's own iteration count
    for that solve at n = 4095 (iteration counts are flat in n).  The sample
    runs on one thread (numpy's convolution and scipy's DST-I are
    single-threaded).  With `all_cores`, the same sample also runs in one
    spawned process per host core at once, since the workload's 60 solves are
    independent: the sum of their rates is the all-cores figure."""
    import oracle
    import workloads
    t, its = oracle_sample(n)
    ws = workloads.var_1d_time_stepping(n=4095, alphas=(1.8,))[0]
    hs = 1.0 / 4096
    ps = oracle.Problem1D(alpha=1.8, n=4095, c0=hs ** 1.8 / ws["dt"], dp=ws["dp"], dm=ws["dm"])
    rs = oracle.gmres(ps.matvec, ps.c0 * ws["u0"], Pinv=oracle.Tau1D.for_problem(ps).apply_inverse,
                      x0=ws["u0"], restart=RESTART, tol=TOL)
    t_solve = t / its * rs.iterations
    out = {"value": 1.0 / t_solve, "unit": "solves/s", "cores": 1, "kind": "oracle",
           "sample": f"{its} GMRES iterations of the first alpha=1.8 solve at n={n} "
                     f"({t:.1f} s, direct Toeplitz sums, single-threaded numpy), scaled by the oracle's "
                     f"{rs.iterations} iterations for that solve at n=4095"}
    if all_cores:
        try:
            out["all_cores"] = all_cores_sample(n, rs.iterations)
        except Exception as e:  # context only; the one-thread figure stands
            out["all_cores"] = {"error": str(e)}
    return out


def all_cores_sample(n: int, its_per_solve: int, timeout_s: float = 300.0, cores: int = 0):
    """oracle_sample in one spawned process per host core at once.  The
    workers' BLAS runs one thread each: with a BLAS thread pool per process,
    the idle pools' spinning threads starve the compute threads of the others
    (a run of 8 such workers had not finished after 15 minutes).  Workers are
    terminated if the samples do not finish within `timeout_s`.  `cores`: 0
    for every host core."""
    import multiprocessing
    cores = cores or os.cpu_count() or 1
    one = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in one}
    os.environ.update({k: "1" for k in one})
    pool = multiprocessing.get_context("spawn").Pool(cores)
    try:
        runs = pool.map_async(oracle_sample, [n] * cores).get(timeout_s)
    finally:
        pool.terminate()
        pool.join()
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return {"value": sum(i / (tp * its_per_solve) for tp, i in runs), "unit": "solves/s", "cores": cores,
            "sample": f"the same sample in {cores} spawned processes at once (one BLAS thread each)"}


def run_reference(args):
    """The oracle on the host cores, same metric and unit (bounded samples)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ts = []
    base = None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        base = cpu_baseline_sample(args.n)
        if i >= args.warmup:
            ts.append(time.perf_counter() - t0)
    line = {"impl": "reference", "metric": "solves/s", "value": base["value"], "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(ts) / len(ts), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"1d-var-n{args.n}-3alpha-20steps-gmres30", "n": args.n},
            "cpu_baseline": base,
            "e2e": {"value": base["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def job_throughput(ms_local: float, units_per_rank: int, world: int, device):
    """Whole-job figures of a weak-scaling run: the slowest rank's time (max
    over ranks) and the units all ranks processed per second.  Every rank
    must call it (a collective when world > 1)."""
    import torch
    ms = float(ms_local)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    return ms, units_per_rank * world / (ms * 1e-3)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if args.only:
        out = run_2d(args, device) if args.only == "2d" else run_batch(args, device, rank, world)
        if rank == 0:
            print(json.dumps({"section": args.only, "results": out}), flush=True)
        return
    res = run_ours(args, rank, world, device)
    batch = run_batch(args, device, rank, world) if args.batch else None
    two_d = run_2d(args, device) if args.two_d else None
    # headline: the fastest precision path with the workload's preconditioner (the
    # paper's P_F) that met relres 1e-8 on every solve; "+variant" paths use other
    # preconditioners and are reported beside it
    good = {k: v for k, v in res.items() if v["converged"] and "+" not in k}
    pool = good or {k: v for k, v in res.items() if "+" not in k}
    head_k = max(pool, key=lambda k: pool[k]["solves_per_s"])
    head = res[head_k]
    n = args.n
    ms, value = job_throughput(head["ms_per_step"], TIME_STEPS * len(ALPHAS), world, device)
    e2e_ms, e2e_value = job_throughput(head["e2e_ms"], TIME_STEPS * len(ALPHAS), world, device)
    if rank == 0:
        bytes_step = len(ALPHAS) * n * 8
        line = {
            "metric": "solves/s", "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if head_k == "f64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": f"1d-var-n{n}-3alpha-20steps-gmres30", "n": n, "alphas": list(ALPHAS),
                       "time_steps": TIME_STEPS, "restart": RESTART, "tol": TOL, "precision": head_k,
                       "batched": "3 alphas per launch", "l2": "flushed (512 MB write) before each step",
                       "teams": "sized by the previous time step's iteration counts" if args.balance
                       else "even split",
                       "launch": "20 time steps replayed as one CUDA graph" if args.graph else "eager"},
            "unknown_iters_per_s": head["unknown_iters_per_s"] * world,
            "iterations_per_step": head["iterations"],
            "worst_relres": head["worst_relres"],
            "e2e": {"value": e2e_value, "unit": "solves/s",
                    "h2d_bytes_per_step": bytes_step, "d2h_bytes_per_step": bytes_step},
            # per time step: one fde_step_rhs per alpha, k_balance when balancing, the engine
            "gpu_launches": (TIME_STEPS * (len(ALPHAS) + 1 + (1 if args.balance else 0))) * args.steps,
            "roofline": head["roofline"], "clocks": head["clocks"],
            "paths": {k: {kk: v[kk] for kk in ("ms_per_step", "solves_per_s", "unknown_iters_per_s", "iterations",
                                                "outer", "worst_relres", "converged", "roofline", "launch_ms",
                                                "schedule")}
                      for k, v in res.items()},
        }
        if batch is not None:
            line["batched_workload"] = batch
        if two_d is not None:
            line["workloads_2d"] = two_d
        if world == 1 and not args.no_cpu_baseline:
            try:
                line["cpu_baseline"] = cpu_baseline_sample(n, all_cores=True)
            except Exception as e:  # the baseline is context; never fail the GPU line
                line["cpu_baseline"] = {"error": str(e)}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
