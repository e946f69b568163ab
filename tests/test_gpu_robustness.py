"""Failure paths and determinism, without faulting the GPU: a bounded
cross-CTA wait that runs out, NaN in the right-hand side, a workspace full
of NaN before assembly (nothing may read memory it has not written), and
bit-identical repeated solves (fixed-order reductions)."""

import numpy as np
import pytest
import torch

import paper_1912_13304_gb300 as fde
import workloads
from test_gpu_ops import to_dev

pytestmark = pytest.mark.gpu


def test_barrier_wait_runs_out_and_reports_timeout(gpu):
    # CTA 0's short wait runs out; CTA 1, waiting on another team's barrier
    # with the full ~2 s bound, must notice the abort flag and return at once
    w = workloads.var_1d_time_stepping(n=1023, alphas=(1.5,))[0]
    plan = fde.Plan.from_workload(w)
    status = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    st = fde.lib().fde_selftest_barrier_timeout(plan.handle, status.data_ptr(), fde._stream(None))
    e1.record()
    assert st == fde.OK
    torch.cuda.synchronize()
    assert status.tolist() == [fde.ETIMEOUT, fde.ETIMEOUT]
    assert e0.elapsed_time(e1) < 200.0, e0.elapsed_time(e1)
    # the plan is usable afterwards
    b = plan.rhs(to_dev(gpu, w["u0"], "f64"))
    info = plan.solve(b, x=to_dev(gpu, w["u0"], "f64"), tol=1e-8)
    assert info["status"] == fde.OK, info


@pytest.mark.parametrize("method", ["gmres", "pcg"])
def test_nan_right_hand_side_reports_nonfinite(gpu, method):
    n = 1023
    w = workloads.const_1d(n=n) if method == "pcg" else workloads.var_1d_time_stepping(n=n, alphas=(1.5,))[0]
    plan = fde.Plan.from_workload(w)
    b = np.random.default_rng(3).uniform(-1, 1, n)
    b[n // 3] = np.nan
    info = plan.solve(to_dev(gpu, b, "f64"), tol=1e-8)
    assert info["status"] == fde.ENONFINITE, info


@pytest.mark.parametrize("case", ["1d-split", "1d-cta", "2d", "ir"])
def test_nan_poisoned_workspace_gives_identical_solves(gpu, case):
    if case == "2d":
        w = workloads.var_2d_time_stepping(n=255, steps=1)
    else:
        w = workloads.var_1d_time_stepping(n=16383 if case != "1d-cta" else 1023, alphas=(1.8,))[0]
    prec = "f32_ir" if case == "ir" else "f64"
    xs = []
    for fill in (None, 0xFF):
        plan = fde.Plan.from_workload(w, precision=prec, workspace_fill=fill)
        u0 = to_dev(gpu, w["u0"], "f64")
        b = plan.rhs(u0)
        info = plan.solve(b, x=u0.clone(), tol=1e-8, inner_tol=1e-4, max_iters=3000, max_outer=100)
        assert info["status"] == fde.OK, (fill, info)
        xs.append(info["x"])
    assert torch.equal(xs[0], xs[1])


def test_repeated_solves_are_bit_identical(gpu):
    ws = workloads.var_1d_time_stepping(n=16383, alphas=(1.2, 1.8))
    plans = [fde.Plan.from_workload(w) for w in ws]
    bs = [p.rhs(to_dev(gpu, w["u0"], "f64")) for p, w in zip(plans, ws)]
    runs = []
    for _ in range(2):
        xs = [to_dev(gpu, w["u0"], "f64") for w in ws]
        infos = fde.solve_batch(plans, bs, xs, tol=1e-8)
        runs.append((xs, [i["iterations"] for i in infos]))
    assert runs[0][1] == runs[1][1]
    for a, b in zip(runs[0][0], runs[1][0]):
        assert torch.equal(a, b)
