"""Benchmark of the tau-preconditioned Krylov solves on one GB300.

Headline workload (one bench "step" = one implicit-Euler time step): the 2D
variable-coefficient FDE on a 4095 x 4095 grid (16.8M unknowns), alpha = 1.3,
beta = 1.8, d+ = 1+x+y, d- = 2-x, e+ = 1+xy, e- = 1+y^2, dt = 1/256, from
u0 = sin(pi x) sin(pi y), GMRES(20) with the 2D tau(F) D_N preconditioner,
true relres 1e-8.  The march has 50 steps: the W warm-up steps are steps
1..W and the K timed steps are steps W+1..W+K, replayed as one CUDA graph
(the default W = 3, K = 47 times exactly the 50-step march).  Both precision
paths are timed (plain FP64; FP32 inner GMRES with FP64 refinement); the
faster one that reaches relres 1e-8 on every step is the headline.

Side sections in the same JSON line: the 1D variable-coefficient march
(n = 65535, three alphas, 20 steps, GMRES(30)), the 1D constant-coefficient
PCG solve (n = 1023, latency), the batch of 256 independent 1D solves, the
2047^2 constant-coefficient PCG solve, and the Crank-Nicolson step of the
4095^2 plane.  Every section states its own roofline, its relative error
against the CPU oracle and the oracle's own time on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own copy of the march (the solves of
different ranks are independent: no collective on the data path, weak
scaling); the 256-instance batch is sharded over the ranks by cost.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TOL = 1e-8
MARCH_STEPS = 50                    # time steps of the 2D headline march
MARCH_1D_STEPS = 20
ALPHAS_1D = (1.2, 1.5, 1.8)
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2
# FP64 ALU peak derived from the unit counts: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP64_PEAK_SOURCE = "derived: 152 SM x 2 DFMA/clk x 2 x 2.07 GHz"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=47)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precisions", default="f64,f32_ir")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the oracle's reference solutions (the relative errors are then not stated)")
    ap.add_argument("--sections", default="march1d,latency1d,batch,const2d,cn2d",
                    help="side sections to time beside the headline (comma-separated; empty for none)")
    ap.add_argument("--only", default="", help="time only this section (headline or a side section) and print it")
    ap.add_argument("--side-steps", type=int, default=3, help="timed repetitions of each side section")
    ap.add_argument("--inner-tol", type=float, default=1e-4,
                    help="relative tolerance of each FP32 inner solve on the 4095^2 planes (the march and the "
                         "Crank-Nicolson step)")
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
# peaks, measured traffic
# ---------------------------------------------------------------------------

def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def hbm_peak() -> tuple[float, str]:
    p = measured_peaks()
    if "hbm_gbs" in p:
        return float(p["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6800.0, "fallback 6.8 TB/s"


def source_hash() -> str:
    """SHA-256 (16 hex digits) of the CUDA sources and the C header: a traffic
    figure taken by ncu applies only to the kernels built from these bytes."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1912_13304_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    with open(os.path.join(ROOT, "include", "fde.h"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(key: str, units: float):
    """DRAM bytes (read + write) of one launch of the dominant kernel for the
    workload `key`, from profiles/traffic.json (written from an ncu capture):
    bytes per unit of work there times `units`, the work of one launch here.
    None when no capture exists or the kernels changed since it was taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tab = json.load(f)
    except Exception:
        return None
    e = tab.get(key)
    if not e or e.get("source_hash") != source_hash():
        return None
    return float(e["dram_bytes"]) / float(e["units"]) * units


# ---------------------------------------------------------------------------
# algorithmic work of a solve, from the device's work counters
# ---------------------------------------------------------------------------

def fft_flops(L: int) -> float:
    """Flops of one real-packed FFT of L real points (an L/2-point complex FFT
    plus the pair step), the 2.5 L log2 L of the split-radix count."""
    return 2.5 * L * math.log2(L)


# Real-packed line transforms per iteration: the tau solve's two sine
# transforms, plus the matvec's forward and one inverse transform (PCG,
# symmetric multiplier) or two inverse transforms (GMRES: D_+ T x and D_- T^T x).
FFTS_PER_ITERATION = {"pcg": 4, "gmres": 5}


class Geometry:
    """What the byte count of one solve depends on: the grid, the method and
    which coefficient arrays a product reads."""

    def __init__(self, dim: int, n1: int, n2: int, method: str, has_D: bool, ncoef: int):
        self.dim, self.n1, self.n2 = dim, n1, (n2 if dim == 2 else 1)
        self.N = n1 * self.n2
        self.method, self.has_D, self.ncoef = method, has_D, ncoef

    @classmethod
    def of_workload(cls, w: dict, method=None, shift=None):
        method = method or w["method"]
        shift = w["shift"] if shift is None else shift
        const = w["const_coeffs"]
        arrays = 0 if const else (2 if w["dim"] == 1 else 4)
        if w["dim"] == 1:
            has_D = not shift or not const
        else:
            has_D = not shift
        return cls(w["dim"], w["n1"], w["n2"], method, has_D, arrays)

    def transform_flops(self) -> float:
        """Flops of the line transforms of one iteration."""
        f = FFTS_PER_ITERATION[self.method]
        if self.dim == 1:
            return f * fft_flops(2 * (self.n1 + 1))
        return f * (self.n2 * fft_flops(2 * (self.n1 + 1)) + self.n1 * fft_flops(2 * (self.n2 + 1)))


def solve_bytes(info: dict, g: Geometry, e_inner: int) -> float:
    """Algorithmic bytes of one solve: every N-vector the method reads or
    writes, once per use, with on-chip transform intermediates (nothing the
    implementation adds -- a second Gram-Schmidt pass, the 2D x/y
    intermediate -- is counted).  e_inner: element bytes of the Krylov
    vectors (8 FP64, 4 FP32); iterations on FP64 vectors (info iterations64)
    count 8 bytes.  Per GMRES step j of a cycle: forming V_j (j >= 1) reads w
    and j basis vectors and writes V_j; the tau solve reads V_j (and D^-1) and
    writes z; the matvec reads z and the coefficient arrays and writes w; the
    dots read w and j+1 basis vectors.  Per cycle: the true residual (a matvec
    that also reads b), its norm, and the update x += P^-1 V y (k basis
    vectors, D^-1, x read and written).  PCG: per iteration the matvec, the
    tau solve, two dots, the norm and three vector updates; per cycle the
    residual, its norm, one tau solve and dot, and p = z.  Refinement: per
    FP64 residual a matvec reading x and b (8 bytes), the norm, the FP32
    right-hand side and zero start, and the update of x."""
    N = g.N
    its, cyc = info["iterations"], max(info["cycles"], 1 if info["iterations"] else 0)
    its64 = info.get("iterations64", 0)
    tau = 2 + (1 if g.has_D else 0)
    mv = 2 + g.ncoef
    if g.method == "gmres":
        sj = info["basis_sum"] - its                 # sum of j over the steps
        passes = (sj + 2 * (its - cyc)) + (sj + 2 * its) + its * (tau + mv)
        passes += cyc * (mv + 1 + 1) + its + cyc * ((1 if g.has_D else 0) + 2)
    else:
        passes = its * (mv + tau + 14) + cyc * (mv + 1 + 1 + tau + 2 + 2)
    frac64 = its64 / its if its else 1.0
    e_eff = 8 * frac64 + e_inner * (1 - frac64)
    b = passes * e_eff * N
    b += info.get("residuals64", 0) * N * ((mv + 2) * 8 + 16 + 20)
    return float(b)


def solve_flops(info: dict, g: Geometry) -> float:
    """Transform flops of one solve: its iterations plus one matvec per cycle
    and FP64 residual and one tau solve per cycle (2/5 and 2/5 of an iteration)."""
    per = g.transform_flops()
    f = FFTS_PER_ITERATION[g.method]
    extra = info["cycles"] * (f - 2 + 2) / f + info.get("residuals64", 0) * (f - 2) / f
    return per * (info["iterations"] + extra)


def roofline_hbm(bytes_, ms, key=None, units=None, launches=1):
    peak, src = hbm_peak()
    achieved = bytes_ / (ms * 1e-3) / 1e9
    traffic = measured_traffic(key, units) if key else None
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "algorithmic_bytes_per_launch": bytes_ / launches, "peak_source": src}


def roofline_alu(flops, ms, fp64_measured=None, key=None, units=None, launches=1):
    achieved = flops / (ms * 1e-3) / 1e12
    out = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
           "frac": achieved / FP64_PEAK_TFLOPS, "traffic": measured_traffic(key, units) if key else None,
           "algorithmic_flops_per_launch": flops / launches, "peak_source": FP64_PEAK_SOURCE}
    if fp64_measured:
        out["peak_measured"] = fp64_measured
        out["frac_of_measured"] = achieved / fp64_measured
    return out


def alu_roofline(flops: float, ms: float, peak_tflops: float) -> dict:
    achieved = flops / (ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": achieved / peak_tflops, "traffic": None, "peak_source": FP64_PEAK_SOURCE}


# ---------------------------------------------------------------------------
# the CPU oracle: reference solutions (relative error per result) and the
# timed CPU baseline.  Module-level functions, so spawned processes run them.
# ---------------------------------------------------------------------------

def _oracle_problem(w: dict, scheme_cn: bool = False):
    import oracle
    n1 = w["n1"]
    h1 = w["length"] / (n1 + 1)
    c0 = (2.0 if scheme_cn else 1.0) * h1 ** w["alpha"] / w["dt"]
    if w["dim"] == 1:
        return oracle.Problem1D(alpha=w["alpha"], n=n1, c0=c0, dp=w["dp"], dm=w["dm"], scheme=w["scheme"])
    h2 = w["length"] / (w["n2"] + 1)
    return oracle.Problem2D(alpha=w["alpha"], beta=w["beta"], n1=n1, n2=w["n2"], c0=c0,
                            sr=h1 ** w["alpha"] / h2 ** w["beta"], dp=w["dp"], dm=w["dm"], ep=w["ep"], em=w["em"],
                            scheme=w["scheme"])


def _oracle_precond(w: dict, prob, shift=None):
    import oracle
    shift = w["shift"] if shift is None else shift
    if w["dim"] == 1:
        P = oracle.Tau1D.for_problem(prob, shift=shift)
        P.fast = True
        return P
    return oracle.Tau2D.for_problem(prob, shift=shift)


def oracle_solve(w: dict, b, x0=None, tol: float = TOL, maxiter: int = 10000):
    """The oracle's textbook solve of one system of workload w (fast operators:
    Toeplitz sums by library-FFT convolution, tau by the library DST-I)."""
    import oracle
    prob = _oracle_problem(w)
    P = _oracle_precond(w, prob)
    A = lambda v: prob.matvec(v, "fft")
    if w["method"] == "pcg":
        return oracle.pcg(A, b, Pinv=P.apply_inverse, x0=x0, tol=tol, maxiter=maxiter)
    return oracle.gmres(A, b, Pinv=P.apply_inverse, x0=x0, restart=w["restart"], tol=tol, maxiter=maxiter)


def oracle_references(workers: int) -> dict:
    """Reference solutions the bench compares its results with, computed by
    the oracle alone (in a spawned process, while the GPU runs):
      march2d:  the first step of the 4095^2 march (tol 1e-8, x0 = u0);
      march1d:  the whole 20-step march of each alpha at n = 65535;
      latency1d: the n = 1023 PCG solve at tol 1e-13;
      const2d:  the 2047^2 PCG solve at tol 1e-13;
      batch:    all 256 instances at tol 1e-13."""
    import numpy as np

    import oracle
    import workloads
    oracle.set_fft_workers(workers)
    out = {}
    t0 = time.perf_counter()
    w = workloads.const_1d()
    prob = _oracle_problem(w)
    r = oracle_solve(w, prob.c0 * w["b"], tol=1e-13, maxiter=500)
    out["latency1d"] = {"x": r.x, "iterations": r.iterations}
    w = workloads.const_2d()
    prob = _oracle_problem(w)
    r = oracle_solve(w, prob.c0 * w["b"], tol=1e-13, maxiter=500)
    out["const2d"] = {"x": r.x, "iterations": r.iterations}
    xs = []
    for w in workloads.const_1d_batch():
        prob = _oracle_problem(w)
        xs.append(oracle_solve(w, prob.c0 * w["b"], tol=1e-13, maxiter=500).x)
    out["batch"] = {"x": xs}
    finals, its = [], []
    for w in workloads.var_1d_time_stepping(n=65535, alphas=ALPHAS_1D, steps=MARCH_1D_STEPS):
        prob = _oracle_problem(w)
        u = w["u0"].copy()
        k = 0
        for _ in range(MARCH_1D_STEPS):
            r = oracle_solve(w, prob.c0 * u, x0=u)
            u = r.x
            k += r.iterations
        finals.append(u)
        its.append(k)
    out["march1d"] = {"x": finals, "iterations": its}
    w = workloads.var_2d_time_stepping(steps=1)
    prob = _oracle_problem(w)
    r = oracle_solve(w, prob.c0 * w["u0"], x0=w["u0"])
    out["march2d"] = {"x": r.x, "iterations": r.iterations}
    out["seconds"] = time.perf_counter() - t0
    return out


def relerr(x, ref) -> float:
    import numpy as np
    x, ref = np.asarray(x, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def cpu_sample(section: str, workers: int, cap: int) -> dict:
    """The oracle as it stands, timed on a bounded sample of one section's
    workload with `workers` FFT threads: (seconds, iterations, solves) of the
    sample.  The caller scales the sample to the section's metric."""
    import numpy as np

    import oracle
    import workloads
    oracle.set_fft_workers(workers)
    if section in ("march2d", "cn2d"):
        w = workloads.var_2d_time_stepping(steps=1)
        prob = _oracle_problem(w)
        b, x0 = prob.c0 * w["u0"], w["u0"]
    elif section == "march1d":
        w = workloads.var_1d_time_stepping(alphas=(1.5,))[0]
        prob = _oracle_problem(w)
        b, x0 = prob.c0 * w["u0"], w["u0"]
    elif section == "latency1d":
        w = workloads.const_1d()
        b, x0 = _oracle_problem(w).c0 * w["b"], None
    elif section == "const2d":
        w = workloads.const_2d()
        b, x0 = _oracle_problem(w).c0 * w["b"], None
    elif section == "batch":
        ws = workloads.const_1d_batch()[:cap]
        t0 = time.perf_counter()
        its = 0
        for w in ws:
            its += oracle_solve(w, _oracle_problem(w).c0 * w["b"]).iterations
        return {"seconds": time.perf_counter() - t0, "iterations": its, "solves": len(ws),
                "unknowns": sum(w["n1"] for w in ws)}
    else:
        raise ValueError(section)
    t0 = time.perf_counter()
    r = oracle_solve(w, b, x0=x0, maxiter=cap)
    return {"seconds": time.perf_counter() - t0, "iterations": max(r.iterations, 1), "solves": 1,
            "unknowns": w["n1"] * w["n2"]}


def cpu_baseline(section: str, gpu_iterations_per_solve: float, cap: int, cores: int) -> dict:
    """Oracle solves/s on the host for one section: a sample capped at `cap`
    Krylov iterations (batch: the first `cap` instances), at one FFT thread
    and at `cores`; a capped sample is scaled per solve by the iteration
    count the GPU path needed (the oracle runs the same algorithm)."""
    out = {"kind": "oracle", "cores": 1}
    for label, k in (("one", 1), ("all", cores)):
        s = cpu_sample(section, k, cap)
        if section == "batch":
            import workloads
            ws = workloads.const_1d_batch()
            cost = sum(batch_cost(w["n1"]) for w in ws) / sum(batch_cost(w["n1"]) for w in ws[:cap])
            sec_per_solve = s["seconds"] * cost / len(ws)
            sample = f"the first {cap} of the 256 instances, full PCG solves ({s['seconds']:.2f} s), scaled by cost"
        elif s["iterations"] >= cap:
            sec_per_solve = s["seconds"] / s["iterations"] * gpu_iterations_per_solve
            sample = (f"{s['iterations']} Krylov iterations of one solve ({s['seconds']:.2f} s), scaled by the "
                      f"{gpu_iterations_per_solve:.1f} iterations per solve of the GPU path")
        else:
            sec_per_solve = s["seconds"]
            sample = f"one full solve ({s['seconds']:.3f} s, {s['iterations']} iterations)"
        rec = {"value": 1.0 / sec_per_solve, "unit": "solves/s", "cores": k,
               "sample": sample + f", FP64 numpy/scipy with {k} FFT thread(s)"}
        if label == "one":
            out.update(rec)
        else:
            out["all_cores"] = rec
    return out


def batch_cost(n: int) -> float:
    """Relative cost of one constant-coefficient PCG solve of size n: the
    Case I shifted preconditioner keeps the iteration count flat in n, so the
    work per solve goes as the line transforms, L log2 L with L = 2(n+1)."""
    L = 2 * (n + 1)
    return L * math.log2(L)


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


# ---------------------------------------------------------------------------
# our arm: timed sections
# ---------------------------------------------------------------------------

def _timed(run, device, world, reps=1, flush=None, pre=None):
    """Device time (ms, CUDA events on the current stream) of each of `reps`
    calls of run(), bracketed by a barrier and synchronisations; `pre()` and,
    if given, a write of `flush` (a buffer larger than L2) run before each
    call, untimed."""
    import torch
    out = []
    for _ in range(reps):
        if pre is not None:
            pre()
        if flush is not None:
            flush.fill_(1.0)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        s0.record()
        run()
        s1.record()
        torch.cuda.synchronize()
        out.append(s0.elapsed_time(s1))
    return out


def _summary(infos):
    return {"iterations": sum(i["iterations"] for i in infos), "outer": sum(i["outer"] for i in infos),
            "reorth": sum(i["reorth"] for i in infos), "worst_relres": max(i["relres"] for i in infos),
            "converged": all(i["status"] == 0 and i["relres"] <= TOL for i in infos)}


def section_march2d(args, device, world, clk_index):
    """Headline: the 4095^2 variable-coefficient march (see the module
    docstring).  Returns per precision path the timed steps' figures and
    the first step's solution (for the oracle comparison)."""
    import torch

    import paper_1912_13304_gb300 as fde
    import workloads
    from paper_1912_13304_gb300.solver import TimeStepper
    w = workloads.var_2d_time_stepping(steps=MARCH_STEPS)
    g = Geometry.of_workload(w)
    N = g.N
    u0 = torch.tensor(w["u0"], dtype=torch.float64, device=device)
    kw = dict(tol=TOL, max_iters=5000, inner_tol=args.inner_tol, max_outer=100, balance=False)
    K, W = args.steps, args.warmup
    paths = {}
    keep = {}
    for prec in [p for p in args.precisions.split(",") if p]:
        plan = fde.Plan.from_workload(w, precision=prec, device=device)
        u = u0.clone()
        one = TimeStepper([plan], [u], 1, graph=False, **kw)
        x1 = None
        for m in range(W):                          # steps 1..W, eager
            one.run()
            if m == 0:
                torch.cuda.synchronize()
                x1 = u.cpu().numpy()
        torch.cuda.synchronize()
        state = u.clone()
        stepper = TimeStepper([plan], [u], K, graph=True, **kw)   # steps W+1..W+K, one graph
        with ClockSampler(clk_index) as clk:
            ms = _timed(stepper.run, device, world, pre=lambda: u.copy_(state))[0]
        infos = [st[0] for st in stepper.infos()]
        s = _summary(infos)
        bytes_ = sum(solve_bytes(i, g, 8 if prec == "f64" else 4) for i in infos)
        flops = sum(solve_flops(i, g) for i in infos)
        rec = dict(ms_per_step=ms / K, solves_per_s=K / (ms * 1e-3), unknown_iters_per_s=N * s["iterations"] /
                   (ms * 1e-3), iterations_per_step=s["iterations"] / K, **s, clocks=clk.summary(),
                   algorithmic_bytes_per_step=bytes_ / K)
        if prec == "f64":
            rec["roofline"] = roofline_alu(flops, ms, args.fp64_measured, key=f"march2d:{prec}",
                                           units=bytes_ / K, launches=K)
            rec["roofline_hbm"] = roofline_hbm(bytes_, ms, key=f"march2d:{prec}", units=bytes_ / K, launches=K)
        else:
            rec["roofline"] = roofline_hbm(bytes_, ms, key=f"march2d:{prec}", units=bytes_ / K, launches=K)
        paths[prec] = rec
        keep[prec] = (plan, u, state, x1)
    # headline path: the fastest that converged on every timed step
    good = [p for p in paths if paths[p]["converged"]] or list(paths)
    head = max(good, key=lambda p: paths[p]["solves_per_s"])
    plan, u, state, _ = keep[head]
    # end to end through the public API: every step copies its input state from
    # pinned host memory and its solution back
    host = torch.empty(N, dtype=torch.float64).pin_memory()

    def e2e():
        for _ in range(K):
            u.copy_(host, non_blocking=True)
            b = plan.rhs(u)
            fde.solve_batch([plan], [b], [u], read_info=False, **kw)
            host.copy_(u, non_blocking=True)

    host.copy_(state)
    e2e_ms = _timed(e2e, device, world)[0]
    paths[head]["e2e_ms_per_step"] = e2e_ms / K
    return {"workload": f"2d-var-n{w['n1']}-50steps-gmres20", "unknowns": N, "head": head, "paths": paths,
            "first_step": {p: keep[p][3] for p in keep}, "e2e_ms": e2e_ms,
            "e2e_bytes_per_step": N * 8}


def kappa_estimate(w: dict) -> float:
    """kappa(M) of a 1D variable-coefficient system from its symbol: the
    largest eigenvalue of the Toeplitz part is at most 2^(alpha+1) max d and
    the smallest at least p_alpha(theta_1) min d, theta_1 = pi/(n+1), with
    p_alpha(theta) = g(theta) + g(-theta), g(theta) = -e^{-i theta}
    (1 - e^{i theta})^alpha (Sec. 2.2), d = (d_+ + d_-)/2 and the identity
    shift nu = h^alpha / dt on both."""
    import numpy as np
    n, a = w["n1"], w["alpha"]
    h = w["length"] / (n + 1)
    nu = h ** a / w["dt"]
    d = 0.5 * (np.asarray(w["dp"], dtype=np.float64) + np.asarray(w["dm"], dtype=np.float64))
    th = math.pi / (n + 1)
    g = lambda t: -np.exp(-1j * t) * np.power(1.0 - np.exp(1j * t), a)
    p1 = float(np.real(g(th) + g(-th)))
    return float((nu + d.max() * 2.0 ** (a + 1)) / (nu + d.min() * p1))


# An FP32 product carries an error of about u32 ||M|| ||x||: relative to the
# smallest eigenmodes that is u32 kappa, and the FP32 inner solves need a
# growing multiple of the FP64 iteration count once it nears 1e-2 (the
# march1d section reports the counts per alpha beside this rule's choice).
U32_KAPPA_LIMIT = 1e-2


def precision_by_alpha(ws, paths):
    """Per alpha of the 1D march: the kappa estimate, u32 kappa, the
    iterations each precision path took, and the precision the u32 kappa
    rule picks (FP32 inner solves only while u32 kappa < U32_KAPPA_LIMIT)."""
    out = {}
    for w in ws:
        a = str(w["alpha"])
        k = kappa_estimate(w)
        its = {p: paths[p]["per_alpha"][a]["iterations"] for p in ("f64", "f32_ir") if p in paths}
        out[a] = {"kappa_estimate": k, "u32_kappa": k * 2.0 ** -24, "iterations": its,
                  "choice": "f32_ir" if k * 2.0 ** -24 < U32_KAPPA_LIMIT else "f64"}
    return out


def section_march1d(args, device, world):
    """The 1D variable-coefficient march (n = 65535, alpha in {1.2, 1.5, 1.8},
    20 implicit-Euler steps, GMRES(30), the three alphas batched in one launch
    per step, teams sized by the previous step's iteration counts, the 20
    steps one CUDA graph); one repetition = the whole march, L2 flushed
    before each.  Paths: FP64, FP32 inner + FP64 outer, and in FP64 the
    shifted variant and P_F-tilde."""
    import torch

    import paper_1912_13304_gb300 as fde
    import workloads
    from paper_1912_13304_gb300.solver import TimeStepper
    ws = workloads.var_1d_time_stepping(n=65535, alphas=ALPHAS_1D, steps=MARCH_1D_STEPS)
    n = ws[0]["n1"]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    u0 = [torch.tensor(w["u0"], dtype=torch.float64, device=device) for w in ws]
    runs = [(p, "") for p in args.precisions.split(",") if p] + [("f64", "shift"), ("f64", "ftilde")]
    out = {}
    finals = {}
    for prec, variant in runs:
        key = prec + ("+" + variant if variant else "")
        plans = [fde.Plan.from_workload(w, precision=prec, shift=variant == "shift",
                                        order="tau_df" if variant == "ftilde" else None, device=device) for w in ws]
        schedule = [p.autotune() for p in plans][0]
        u = [x.clone() for x in u0]
        kw = dict(tol=TOL, max_iters=20000, inner_tol=1e-3, max_outer=200, balance=True)
        stepper = TimeStepper(plans, u, MARCH_1D_STEPS, graph=True, **kw)

        def reset():
            for k in range(len(ws)):
                u[k].copy_(u0[k])

        for _ in range(max(1, args.warmup)):
            reset()
            stepper.run()
        torch.cuda.synchronize()
        ms = _timed(stepper.run, device, world, reps=args.side_steps, flush=flush, pre=reset)
        t = sum(ms) / len(ms)
        infos = [i for st in stepper.infos() for i in st]
        s = _summary(infos)
        g = Geometry.of_workload(ws[0], shift=variant == "shift")
        bytes_ = sum(solve_bytes(i, g, 8 if prec == "f64" else 4) for i in infos)
        flops = sum(solve_flops(i, g) for i in infos)
        nsolves = MARCH_1D_STEPS * len(ws)
        rec = dict(ms_per_march=t, solves_per_s=nsolves / (t * 1e-3), unknown_iters_per_s=n * s["iterations"] /
                   (t * 1e-3), **s, schedule={"ctas": schedule[0], "log_p1": schedule[1]})
        rec["per_alpha"] = {str(w["alpha"]): {"iterations": sum(st[k]["iterations"] for st in stepper.infos()),
                                              "outer": sum(st[k]["outer"] for st in stepper.infos())}
                            for k, w in enumerate(ws)}
        if prec == "f64":
            rec["roofline"] = roofline_alu(flops, t, args.fp64_measured, key=f"march1d:{key}",
                                           units=bytes_ / MARCH_1D_STEPS, launches=MARCH_1D_STEPS)
        else:
            rec["roofline"] = roofline_hbm(bytes_, t, key=f"march1d:{key}", units=bytes_ / MARCH_1D_STEPS,
                                           launches=MARCH_1D_STEPS)
        out[key] = rec
        finals[key] = [x.cpu().numpy() for x in u]
        for p in plans:
            p.close()
    return {"workload": f"1d-var-n{n}-3alpha-20steps-gmres30", "unknowns": n, "paths": out, "finals": finals,
            "precision_by_alpha": precision_by_alpha(ws, out)}


def section_latency1d(args, device, world):
    """The 1D constant-coefficient solve (n = 1023, alpha = 1.5, d = 1,
    dt = h, PCG with the Case I shifted tau preconditioner, relres 1e-8): a
    latency figure, microseconds per solve, from a CUDA graph of 100 solves
    (each from x = 0, one launch each)."""
    import torch

    import paper_1912_13304_gb300 as fde
    import workloads
    w = workloads.const_1d()
    g = Geometry.of_workload(w)
    reps = 100
    out = {}
    xs = {}
    for prec in [p for p in args.precisions.split(",") if p]:
        plan = fde.Plan.from_workload(w, precision=prec, device=device)
        # the autotuner picks between one CTA per line and a line split over a
        # team of CTAs (at FP64 one SM's pipe makes the single-CTA line slow)
        schedule = plan.autotune()
        b = plan.c0 * torch.tensor(w["b"], dtype=torch.float64, device=device)
        x = torch.zeros_like(b)
        info = torch.zeros(fde.INFO_BYTES, dtype=torch.uint8, device=device)
        kw = dict(tol=TOL, max_iters=500, inner_tol=1e-5, max_outer=50, info_dev=info, read_info=False)

        def once():
            x.zero_()
            fde.solve_batch([plan], [b], [x], **kw)

        for _ in range(3):
            once()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for _ in range(reps):
                once()
        ms = _timed(graph.replay, device, world, reps=max(1, args.side_steps))
        t = sum(ms) / len(ms) / reps
        inf = fde.decode_info(info.cpu().numpy().tobytes(), 1)[0]
        s = _summary([inf])
        rec = dict(us_per_solve=1e3 * t, solves_per_s=1.0 / (t * 1e-3), **s,
                   schedule={"ctas": schedule[0], "log_p1": schedule[1]},
                   unknown_iters_per_s=w["n1"] * inf["iterations"] / (t * 1e-3),
                   algorithmic_bytes_per_solve=solve_bytes(inf, g, 8 if prec == "f64" else 4))
        # the working set (~100 KB) lives in one SM's shared memory and L1: a
        # latency, not a bandwidth, figure; the FP64 flop rate is stated
        rec["roofline"] = roofline_alu(solve_flops(inf, g), t, args.fp64_measured)
        out[prec] = rec
        xs[prec] = x.cpu().numpy()
        plan.close()
    return {"workload": f"1d-const-n{w['n1']}-pcg-case1", "unknowns": w["n1"], "paths": out, "x": xs}


def batch_job(local: dict, world: int, device) -> dict:
    """Whole-job figures of the sharded batch (every rank calls it; a
    collective when world > 1): the slowest rank's launch time, the worst
    relres and per-size iteration maximum, summed iterations, bytes, flops and
    unknown-iterations, and whether every rank converged.  `max_its_by_k`
    holds one entry per k of BATCH_KS (0 where a rank has no such size)."""
    if world == 1:
        return dict(local)
    import torch
    mx = torch.tensor([local["ms_per_launch"], local["worst_relres"]] + list(local["max_its_by_k"]),
                      dtype=torch.float64, device=device)
    sm = torch.tensor([local["iterations"], local["outer"], local["unknown_iters"], local["flops"],
                       local.get("bytes", 0.0), 0.0 if local["converged"] else 1.0], dtype=torch.float64,
                      device=device)
    torch.distributed.all_reduce(mx, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(sm, op=torch.distributed.ReduceOp.SUM)
    return {"ms_per_launch": float(mx[0]), "worst_relres": float(mx[1]),
            "max_its_by_k": [int(v) for v in mx[2:].tolist()], "iterations": int(sm[0]), "outer": int(sm[1]),
            "unknown_iters": float(sm[2]), "flops": float(sm[3]), "bytes": float(sm[4]),
            "converged": float(sm[5]) == 0.0}


BATCH_KS = range(8, 15)        # n = 2^k - 1 of the batched workload


def section_batch(args, device, rank, world):
    """The batched workload: 256 independent 1D constant-coefficient solves
    (n = 2^k - 1, k ~ U{8..14}; alpha ~ U(1.1, 1.9); d, dt per instance; seed
    2), PCG with each instance's shifted tau preconditioner, relres 1e-8, all
    in one persistent launch.  The figures count the 256 plans' symbol
    assembly too (fde_assemble_symbol of every instance, then the solve
    launch), beside the launch alone.  Under torchrun the instances are
    sharded over the ranks by cost (strong scaling; the results meet in two
    all-reduces of a few scalars)."""
    import torch

    import paper_1912_13304_gb300 as fde
    import workloads
    ws_all = workloads.const_1d_batch()
    mine = shard_by_cost([batch_cost(w["n1"]) for w in ws_all], world)[rank]
    ws = [ws_all[i] for i in mine]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    out = {}
    xs_out = {}
    for prec in [p for p in args.precisions.split(",") if p]:
        plans = [fde.Plan.from_workload(w, precision=prec, device=device) for w in ws]
        bs = [p.c0 * torch.tensor(w["b"], dtype=torch.float64, device=device) for p, w in zip(plans, ws)]
        xs = [torch.zeros_like(b) for b in bs]
        info = torch.zeros(len(ws) * fde.INFO_BYTES, dtype=torch.uint8, device=device)
        kw = dict(tol=TOL, max_iters=2000, inner_tol=1e-4, max_outer=100, info_dev=info, read_info=False)

        def zero():
            for x in xs:
                x.zero_()

        def solve():
            fde.solve_batch(plans, bs, xs, **kw)

        for _ in range(max(1, args.warmup)):
            zero()
            solve()
        torch.cuda.synchronize()
        ms = _timed(solve, device, world, reps=args.side_steps, flush=flush, pre=zero)
        # assembly + solve: the plans' symbol data rebuilt first (the same device
        # kernels fde_assemble_symbol launches), the plans spread over side
        # streams that join the timed stream before the solve launch
        from paper_1912_13304_gb300.solver import reassemble_all
        ms_asm = _timed(lambda: (reassemble_all(plans), solve()), device, world,
                        reps=args.side_steps, flush=flush, pre=zero)
        infos = fde.decode_info(info.cpu().numpy().tobytes(), len(ws))
        max_its = {k: 0 for k in BATCH_KS}
        for w, i in zip(ws, infos):
            k = int(round(math.log2(w["n1"] + 1)))
            max_its[k] = max(max_its[k], i["iterations"])
        geos = [Geometry.of_workload(w) for w in ws]
        job = batch_job({"ms_per_launch": sum(ms) / len(ms),
                         "worst_relres": max((i["relres"] for i in infos), default=0.0),
                         "max_its_by_k": [max_its[k] for k in BATCH_KS],
                         "iterations": sum(i["iterations"] for i in infos),
                         "outer": sum(i["outer"] for i in infos),
                         "unknown_iters": float(sum(w["n1"] * i["iterations"] for w, i in zip(ws, infos))),
                         "flops": sum(solve_flops(i, gg) for i, gg in zip(infos, geos)),
                         "bytes": sum(solve_bytes(i, gg, 8 if prec == "f64" else 4) for i, gg in zip(infos, geos)),
                         "converged": all(i["status"] == 0 and i["relres"] <= TOL for i in infos)},
                        world, device)
        t_asm = job_throughput(sum(ms_asm) / len(ms_asm), 0, world, device)[0]
        t = job["ms_per_launch"]
        rec = {"ms_per_launch": t, "solves_per_s": len(ws_all) / (t * 1e-3),
               "ms_with_assembly": t_asm, "solves_per_s_with_assembly": len(ws_all) / (t_asm * 1e-3),
               "max_iterations_by_n": {str(2 ** k - 1): v for k, v in zip(BATCH_KS, job["max_its_by_k"]) if v > 0},
               "unknown_iters_per_s": job["unknown_iters"] / (t * 1e-3), "iterations": job["iterations"],
               "outer": job["outer"], "worst_relres": job["worst_relres"], "converged": job["converged"]}
        if prec == "f64":
            rec["roofline"] = roofline_alu(job["flops"], t, args.fp64_measured)
        else:
            rec["roofline"] = roofline_hbm(job["bytes"], t)
        out[prec] = rec
        xs_out[prec] = {i: x.cpu().numpy() for i, x in zip(mine, xs)}
        for p in plans:
            p.close()
    return {"workload": "batch256-1d-const-n255..16383-pcg-shifted-tau", "instances": len(ws_all),
            "unknowns": sum(w["n1"] for w in ws_all), "paths": out, "x": xs_out,
            "sharding": "one launch" if world == 1 else f"cost-balanced over {world} ranks (strong scaling)"}


def section_plane(args, device, world, which: str):
    """One solve per repetition on a full plane: `const2d` is the 2047^2
    constant-coefficient system (alpha 1.5, beta 1.7, PCG with P_hat, rhs
    seed 1); `cn2d` is one Crank-Nicolson step of the 4095^2 variable-
    coefficient plane, the explicit half b = (2 c0 I - M) u0 included in the
    timed step (GMRES(20) with tau(F) D_N)."""
    import torch

    import paper_1912_13304_gb300 as fde
    import workloads
    if which == "const2d":
        w = workloads.const_2d()
    else:
        w = dict(workloads.var_2d_time_stepping(steps=1), time_scheme="cn")
    g = Geometry.of_workload(w)
    N = g.N
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    reps = args.side_steps if which == "const2d" else 1
    out, xs = {}, {}
    for prec in [p for p in args.precisions.split(",") if p]:
        if which == "cn2d":
            plan = fde.Plan(2, w["n1"], w["alpha"], w["dt"], n2=w["n2"], beta=w["beta"], len1=w["length"],
                            len2=w["length"], scheme="cn", weights=w["scheme"], dp=w["dp"].reshape(-1),
                            dm=w["dm"].reshape(-1), ep=w["ep"].reshape(-1), em=w["em"].reshape(-1),
                            method="gmres", restart=w["restart"], precision=prec, device=device)
            x0 = torch.tensor(w["u0"], dtype=torch.float64, device=device)
            b = torch.empty_like(x0)
        else:
            plan = fde.Plan.from_workload(w, precision=prec, device=device)
            b = plan.c0 * torch.tensor(w["b"], dtype=torch.float64, device=device)
            x0 = torch.zeros_like(b)
        x = torch.empty_like(x0)
        info = torch.zeros(fde.INFO_BYTES, dtype=torch.uint8, device=device)
        itol = 1e-4 if which == "const2d" else args.inner_tol
        kw = dict(tol=TOL, max_iters=5000, inner_tol=itol, max_outer=100, info_dev=info, read_info=False)

        def step():
            if which == "cn2d":
                plan.rhs(x0, b=b)
            fde.solve_batch([plan], [b], [x], **kw)

        x.copy_(x0)
        step()
        torch.cuda.synchronize()
        ms = _timed(step, device, world, reps=reps, flush=flush, pre=lambda: x.copy_(x0))
        t = sum(ms) / len(ms)
        inf = fde.decode_info(info.cpu().numpy().tobytes(), 1)[0]
        s = _summary([inf])
        bytes_ = solve_bytes(inf, g, 8 if prec == "f64" else 4)
        rec = dict(ms_per_solve=t, solves_per_s=1e3 / t, unknown_iters_per_s=N * inf["iterations"] / (t * 1e-3),
                   **s, relres=inf["relres"])
        if prec == "f64":
            rec["roofline"] = roofline_alu(solve_flops(inf, g), t, args.fp64_measured, key=f"{which}:{prec}",
                                           units=bytes_)
            rec["roofline_hbm"] = roofline_hbm(bytes_, t, key=f"{which}:{prec}", units=bytes_)
        else:
            rec["roofline"] = roofline_hbm(bytes_, t, key=f"{which}:{prec}", units=bytes_)
        out[prec] = rec
        xs[prec] = x.cpu().numpy() if which == "const2d" else None
        plan.close()
        del x, b, x0
        torch.cuda.empty_cache()
    name = "2d-const-n2047-pcg-phat" if which == "const2d" else "2d-var-n4095-gmres20-crank-nicolson-step"
    return {"workload": name, "unknowns": N, "paths": out, "x": xs}


def fp64_rate(device) -> float | None:
    """Measured FP64 FMA rate of this GPU (TFLOP/s) from the library's
    DFMA-chain probe (fde_measure_fp64_rate); None if it is unavailable."""
    try:
        import paper_1912_13304_gb300 as fde
        return fde.measure_fp64_rate()
    except Exception:
        return None


# ---------------------------------------------------------------------------
# the reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_iterations_per_step(n: int = 511) -> int:
    """The oracle's GMRES(20) iterations for the first step of the 2D march on
    an n x n grid (iteration counts under P_F are nearly flat in n)."""
    import workloads
    w = workloads.var_2d_time_stepping(n=n, steps=1)
    prob = _oracle_problem(w)
    return oracle_solve(w, prob.c0 * w["u0"], x0=w["u0"]).iterations


def headline_config(args) -> dict:
    """The headline workload as both arms name it: the 4095^2 march, the
    steps timed, and how L2 is treated between them."""
    return {"workload": "2d-var-n4095-50steps-gmres20", "grid": "4095x4095", "unknowns": 4095 * 4095,
            "alpha": 1.3, "beta": 1.8, "dt": 1 / 256, "restart": 20, "tol": TOL,
            "march": f"steps {args.warmup + 1}..{args.warmup + args.steps} of the {MARCH_STEPS}-step "
                     f"implicit-Euler march",
            "l2": "no flush: the working set (1.5-3 GB of Krylov vectors) exceeds the 129 MB L2"}


def run_reference(args):
    """The oracle on the host cores, on the headline's workload, metric and
    unit: each step one bounded sample (the first step of the 4095^2 march,
    GMRES(20) capped at 2 iterations, all host cores for the library FFTs),
    scaled per solve by the oracle's iteration count for that step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    its = oracle_iterations_per_step()
    ts, vals = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        s = cpu_sample("march2d", cores, 2)
        if i >= args.warmup:
            ts.append(time.perf_counter() - t0)
            vals.append(s["iterations"] / (s["seconds"] * its))
    value = sum(vals) / len(vals)
    base = {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"2 GMRES(20) iterations of the first step of the 4095^2 march per bench step, scaled by the "
                      f"oracle's {its} iterations for that step (at 511^2; flat in n), FP64 numpy/scipy, "
                      f"{cores} FFT threads"}
    line = {"impl": "reference", "metric": "solves/s", "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(ts) / len(ts), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": headline_config(args),
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# main
# ---------------------------------------------------------------------------

def _errors(sec: str, res: dict, refs: dict) -> None:
    """Relative 2-norm error of each path's result against the oracle's
    reference solution, written into the section's paths."""
    if not refs or sec not in refs:
        return
    r = refs[sec]
    for p, rec in res["paths"].items():
        try:
            if sec == "march2d":
                rec["relerr_vs_oracle"] = relerr(res["first_step"][p], r["x"])
                rec["relerr_note"] = "step 1 against the oracle's step 1, both at relres 1e-8"
            elif sec == "march1d":
                rec["relerr_vs_oracle"] = max(relerr(a, b) for a, b in zip(res["finals"][p], r["x"]))
                rec["relerr_note"] = "state after 20 steps, worst alpha, both marches at relres 1e-8 per step"
            elif sec == "batch":
                rec["relerr_vs_oracle"] = max(relerr(x, r["x"][i]) for i, x in res["x"][p].items())
                rec["relerr_note"] = "worst instance at relres 1e-8 against the oracle at 1e-13"
            else:
                rec["relerr_vs_oracle"] = relerr(res["x"][p], r["x"])
                rec["relerr_note"] = "relres 1e-8 against the oracle at 1e-13"
        except Exception as e:
            rec["relerr_vs_oracle"] = None
            rec["relerr_note"] = f"unavailable: {e}"


def _strip(res: dict) -> dict:
    return {k: v for k, v in res.items() if k not in ("first_step", "finals", "x")}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # the oracle's reference solutions, in a spawned process that runs while the GPU is timed
    pool = ref_job = None
    if rank == 0 and not args.no_oracle_check:
        import multiprocessing
        pool = multiprocessing.get_context("spawn").Pool(1)
        ref_job = pool.apply_async(oracle_references, (max(1, (os.cpu_count() or 2) - 2),))
    if world > 1:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    import paper_1912_13304_gb300 as fde
    from paper_1912_13304_gb300 import build as fbuild
    fbuild.build()
    fde.lib()
    args.fp64_measured = fp64_rate(device)
    clk_index = torch.cuda.current_device()
    sections = [s for s in args.sections.split(",") if s]
    if args.only:
        sections = [args.only] if args.only != "march2d" else []
    head = section_march2d(args, device, world, clk_index) if args.only in ("", "march2d") else None
    side = {}
    for sec in sections:
        if sec == "march1d":
            side[sec] = section_march1d(args, device, world)
        elif sec == "latency1d":
            side[sec] = section_latency1d(args, device, world)
        elif sec == "batch":
            side[sec] = section_batch(args, device, rank, world)
        elif sec in ("const2d", "cn2d"):
            side[sec] = section_plane(args, device, world, sec)
    refs = {}
    if ref_job is not None:
        try:
            refs = ref_job.get(timeout=900)
        except Exception as e:
            refs = {"error": str(e)}
        pool.terminate()
        pool.join()
    if head is not None:
        _errors("march2d", head, refs)
    for sec, res in side.items():
        _errors(sec, res, refs)
    # CPU baselines (rank 0, N = 1), after the reference process has finished
    cores = os.cpu_count() or 1
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        caps = {"march2d": 2, "march1d": 6, "latency1d": 500, "batch": 16, "const2d": 2, "cn2d": 2}
        for sec, res in ([("march2d", head)] if head else []) + list(side.items()):
            try:
                p0 = next(iter(res["paths"].values()))
                its = p0.get("iterations_per_step") or p0["iterations"] / (
                    MARCH_1D_STEPS * len(ALPHAS_1D) if sec == "march1d" else 1)
                res["cpu_baseline"] = cpu_baseline(sec, float(its), caps[sec], cores)
            except Exception as e:
                res["cpu_baseline"] = {"error": str(e)}
    if head is None:
        if rank == 0:
            print(json.dumps({"section": args.only, "results": {k: _strip(v) for k, v in side.items()}},
                             default=float), flush=True)
        return
    hp = head["paths"][head["head"]]
    K = args.steps
    ms, value = job_throughput(hp["ms_per_step"] * K, K, world, device)
    e2e_ms, e2e_value = job_throughput(head["e2e_ms"], K, world, device)
    if rank == 0:
        line = {
            "metric": "solves/s", "value": value, "unit": "solves/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if head["head"] == "f64" else "f32+f64", "data": "synthetic",
            "config": headline_config(args),
            "precision": head["head"], "launch": f"the {K} timed steps replayed as one CUDA graph",
            "unknown_iters_per_s": hp["unknown_iters_per_s"] * world,
            "iterations_per_step": hp["iterations_per_step"],
            "worst_relres": hp["worst_relres"],
            "relerr_vs_oracle": hp.get("relerr_vs_oracle"),
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": head["e2e_bytes_per_step"],
                    "d2h_bytes_per_step": head["e2e_bytes_per_step"]},
            # per timed step: fde_step_rhs's kernel and the persistent engine
            "gpu_launches": 2 * K,
            "roofline": hp["roofline"], "clocks": hp["clocks"],
            "fp64_peak_measured_tflops": args.fp64_measured,
            "paths": head["paths"],
            "source_hash": source_hash(),
        }
        if "cpu_baseline" in head:
            line["cpu_baseline"] = head["cpu_baseline"]
        line["sections"] = {k: _strip(v) for k, v in side.items()}
        if refs.get("seconds"):
            line["oracle_reference_seconds"] = refs["seconds"]
        print(json.dumps(line, default=float), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
