"""Oracle parity of the solves at the workloads' full sizes, through the C ABI.

The oracle runs the same textbook PCG / GMRES(m) with its operators in their
fast form (Toeplitz sums as library-FFT convolutions, tau through the library
DST-I; both pinned to the dense definitions by the CPU tests), so that a
16.8M-unknown solve finishes in tens of seconds on the host.

  * 2047^2 constant coefficients, PCG with P_hat (Sec. 3.2): iterations within
    +-1 of the oracle's at 1e-8; at a tight tolerance the FP64 and the
    FP32-inner/FP64-outer solutions agree with the oracle's to 1e-8.
  * 4095^2 variable coefficients, one implicit-Euler step, GMRES(20) with the
    2D tau(F) D_N: iterations within +-1 (FP64); every path's true residual
    recomputed by the oracle.
  * n = 65535 variable coefficients, the first implicit-Euler step, GMRES(30)
    with tau(F) D: iterations within +-1 (FP64).

At tolerance 1e-8 the solutions themselves may differ by up to kappa(M) 1e-8
(the paper's systems reach kappa ~ 1e7 in 1D), so those cases compare
iteration counts and residuals, and the tight cases compare solutions.
"""

import os

import numpy as np
import pytest

import oracle
import paper_1912_13304_gb300 as fde
import workloads
from test_gpu_ops import rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _host_threads():
    oracle.set_fft_workers(os.cpu_count() or 1)
    yield
    oracle.set_fft_workers(1)


def problem_2d(w):
    n1, n2 = w["n1"], w["n2"]
    h1, h2 = w["length"] / (n1 + 1), w["length"] / (n2 + 1)
    return oracle.Problem2D(alpha=w["alpha"], beta=w["beta"], n1=n1, n2=n2, c0=h1 ** w["alpha"] / w["dt"],
                            sr=h1 ** w["alpha"] / h2 ** w["beta"], dp=w["dp"], dm=w["dm"], ep=w["ep"],
                            em=w["em"], scheme=w["scheme"])


def relres(prob, b, x):
    return float(np.linalg.norm(b - prob.matvec(x, "fft")) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def config3():
    w = workloads.const_2d()
    prob = problem_2d(w)
    b = prob.c0 * w["b"]
    P = oracle.Tau2D.for_problem(prob, shift=True)
    A = lambda v: prob.matvec(v, "fft")
    ref = oracle.pcg(A, b, Pinv=P.apply_inverse, tol=1e-8)
    tight = oracle.pcg(A, b, Pinv=P.apply_inverse, tol=1e-13, maxiter=300)
    return w, prob, b, ref, tight


@pytest.mark.parametrize("precision", ["f64", "f32_ir"])
def test_config3_2047_pcg_phat_matches_oracle(gpu, config3, precision):
    w, prob, b, ref, tight = config3
    assert ref.converged and tight.converged
    plan = fde.Plan.from_workload(w, precision=precision)
    info = plan.solve(to_dev(gpu, b, "f64"), tol=1e-8, inner_tol=1e-4, max_outer=100)
    assert info["status"] == fde.OK, info
    if precision == "f64":
        assert abs(info["iterations"] - ref.iterations) <= 1, (info, ref.iterations)
    rr = relres(prob, b, info["x"].cpu().numpy())
    assert rr <= 1.01e-8 and abs(rr - info["relres"]) <= 1e-2 * rr + 1e-12, (rr, info)
    tol = 1e-13 if precision == "f64" else 1e-12
    info2 = plan.solve(to_dev(gpu, b, "f64"), tol=tol, max_iters=300, inner_tol=1e-4, max_outer=100)
    assert info2["status"] == fde.OK, info2
    assert rel_err(info2["x"].cpu().numpy(), tight.x) < 1e-8
    plan.close()


@pytest.fixture(scope="module")
def config5():
    w = workloads.var_2d_time_stepping(steps=1)
    prob = problem_2d(w)
    b = prob.c0 * w["u0"]
    P = oracle.Tau2D.for_problem(prob)
    ref = oracle.gmres(lambda v: prob.matvec(v, "fft"), b, Pinv=P.apply_inverse, x0=w["u0"], restart=20,
                       tol=1e-8)
    return w, prob, b, ref


@pytest.mark.parametrize("precision", ["f64", "f32_ir"])
def test_config5_4095_gmres20_step_matches_oracle(gpu, config5, precision):
    w, prob, b, ref = config5
    assert ref.converged
    plan = fde.Plan.from_workload(w, precision=precision)
    info = plan.solve(to_dev(gpu, b, "f64"), x=to_dev(gpu, w["u0"], "f64"), tol=1e-8, inner_tol=1e-4,
                      max_outer=100)
    assert info["status"] == fde.OK, info
    if precision == "f64":
        assert abs(info["iterations"] - ref.iterations) <= 1, (info, ref.iterations)
    rr = relres(prob, b, info["x"].cpu().numpy())
    # two FP64 evaluations of the residual differ by rounding of order
    # u ||M|| ||x|| / ||b||, about 1e-13 here
    assert rr <= 1.01e-8 and abs(rr - info["relres"]) <= 1e-2 * rr + 1e-12, (rr, info)
    plan.close()


@pytest.mark.parametrize("alpha", [1.2, 1.8])
def test_config2_65535_first_step_matches_oracle(gpu, alpha):
    w = workloads.var_1d_time_stepping(alphas=(alpha,))[0]
    n = w["n1"]
    h = 1.0 / (n + 1)
    prob = oracle.Problem1D(alpha=alpha, n=n, c0=h ** alpha / w["dt"], dp=w["dp"], dm=w["dm"])
    b = prob.c0 * w["u0"]
    ref = oracle.gmres(lambda v: prob.matvec(v, "fft"), b, Pinv=oracle.Tau1D.for_problem(prob).apply_inverse,
                       x0=w["u0"], restart=30, tol=1e-8)
    assert ref.converged
    plan = fde.Plan.from_workload(w)
    info = plan.solve(to_dev(gpu, b, "f64"), x=to_dev(gpu, w["u0"], "f64"), tol=1e-8)
    assert info["status"] == fde.OK, info
    assert abs(info["iterations"] - ref.iterations) <= 1, (info, ref.iterations)
    x = info["x"].cpu().numpy()
    rr = np.linalg.norm(b - prob.matvec(x, "fft")) / np.linalg.norm(b)
    # at kappa(M) ~ 1e7 two FP64 evaluations of the residual differ by about
    # u ||M|| ||x|| / ||b|| ~ 1e-9
    assert rr <= 1.01e-8 and abs(rr - info["relres"]) <= 2e-9, (rr, info)
    plan.close()
