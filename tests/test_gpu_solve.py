"""Parity of the device-resident Krylov solves (fde_krylov_solve) with the
oracle's textbook PCG / GMRES(m) on the same seeded inputs.

Criteria: iteration counts within +-1 of the oracle's at the same tolerance;
solutions compared with a tightly converged oracle solution (relres 1e-12):
relative max-norm error 1e-8 for FP64 and FP32-inner/FP64-outer refinement,
1e-6 for the pure FP32 inner solve; the true residual reported by the device
is re-checked with the oracle's matvec.
"""

import numpy as np
import pytest

import oracle
import paper_1912_13304_gb300 as fde
import workloads
from test_gpu_ops import make_1d, make_2d, rel_err, to_dev

pytestmark = pytest.mark.gpu


def oracle_problem_1d(w):
    n = w["n1"]
    h = w["length"] / (n + 1)
    return oracle.Problem1D(alpha=w["alpha"], n=n, c0=h ** w["alpha"] / w["dt"], dp=w["dp"], dm=w["dm"],
                            scheme=w["scheme"])


@pytest.mark.parametrize("precision", ["f64", "f32_ir"])
@pytest.mark.parametrize("n", [1, 7, 63, 1023, 4095])
def test_pcg_case1_matches_oracle(gpu, n, precision):
    w = workloads.const_1d(n=n)
    prob = oracle_problem_1d(w)
    b = prob.c0 * w["b"]                  # the workload writes (I + dt h^-a (...)) u = b
    P = oracle.Tau1D.for_problem(prob, shift=True)
    ref = oracle.pcg(prob.matvec, b, Pinv=P.apply_inverse, tol=1e-8)
    tight = oracle.pcg(prob.matvec, b, Pinv=P.apply_inverse, tol=1e-13, maxiter=500)
    plan = fde.Plan.from_workload(w, precision=precision)
    info = plan.solve(to_dev(gpu, b, "f64"), tol=1e-8, inner_tol=1e-5)
    x = info["x"].cpu().numpy()
    assert info["status"] == fde.OK, info
    if precision == "f64":
        assert abs(info["iterations"] - ref.iterations) <= 1, (info, ref.iterations)
    assert info["relres"] <= 1e-8
    assert np.linalg.norm(b - prob.matvec(x)) / np.linalg.norm(b) <= 1.01e-8
    info2 = plan.solve(to_dev(gpu, b, "f64"), tol=1e-13, max_iters=500, inner_tol=1e-5)
    assert rel_err(info2["x"].cpu().numpy(), tight.x) < 1e-8


@pytest.mark.parametrize("alpha", [1.2, 1.8])
@pytest.mark.parametrize("n", [63, 1023, 4095, 16383])
def test_gmres_right_variable_coefficients(gpu, n, alpha):
    w = workloads.var_1d_time_stepping(n=n, alphas=(alpha,))[0]
    prob = oracle_problem_1d(w)
    b = prob.c0 * w["u0"]
    P = oracle.Tau1D.for_problem(prob)
    ref = oracle.gmres(prob.matvec, b, Pinv=P.apply_inverse, x0=w["u0"], restart=30, tol=1e-8)
    plan = fde.Plan.from_workload(w)
    info = plan.solve(to_dev(gpu, b, "f64"), x=to_dev(gpu, w["u0"], "f64"), tol=1e-8)
    assert info["status"] == fde.OK, info
    assert abs(info["iterations"] - ref.iterations) <= 1, (info, ref.iterations)
    x = info["x"].cpu().numpy()
    assert np.linalg.norm(b - prob.matvec(x)) / np.linalg.norm(b) <= 1.01e-8
    # 1e-12 lies below the FP64 residual floor at alpha = 1.8 (kappa(M) ~ 1e6):
    # the reference stops on its Arnoldi estimate, the device on its iteration cap
    tight = oracle.gmres(prob.matvec, b, Pinv=P.apply_inverse, restart=30, tol=1e-12, maxiter=3000,
                         stop_on_estimate=True)
    info2 = plan.solve(to_dev(gpu, b, "f64"), tol=1e-12, max_iters=600)
    assert rel_err(info2["x"].cpu().numpy(), tight.x) < 1e-8


@pytest.mark.parametrize("alpha", [1.2, 1.8])
@pytest.mark.parametrize("n", [1023, 16383])
def test_gmres_shifted_variable_coefficients(gpu, n, alpha):
    # the shifted variant on the variable-coefficient workload: iterations
    # within +-1 of the oracle's and far fewer than the unshifted P_F's
    w = workloads.var_1d_time_stepping(n=n, alphas=(alpha,))[0]
    prob = oracle_problem_1d(w)
    b = prob.c0 * w["u0"]
    ref = oracle.gmres(prob.matvec, b, Pinv=oracle.Tau1D.for_problem(prob, shift=True).apply_inverse, x0=w["u0"],
                       restart=30, tol=1e-8)
    plan = fde.Plan.from_workload(w, shift=True)
    info = plan.solve(to_dev(gpu, b, "f64"), x=to_dev(gpu, w["u0"], "f64"), tol=1e-8)
    assert info["status"] == fde.OK, info
    assert abs(info["iterations"] - ref.iterations) <= 1, (info["iterations"], ref.iterations)
    x = info["x"].cpu().numpy()
    assert np.linalg.norm(b - prob.matvec(x)) / np.linalg.norm(b) <= 1.01e-8


# (16383, 1e-12) is left out: there the FP64 evaluation of the true residual
# itself carries rounding of order u ||M|| ||x|| / ||b|| ~ 1e-11, so whether a
# cycle's residual passes 1e-12 depends on rounding order alone
@pytest.mark.parametrize("n,tol", [(255, 1e-10), (255, 1e-12), (4095, 1e-10), (4095, 1e-12), (16383, 1e-10)])
def test_gmres_right_tight_tolerance_iterations(gpu, n, tol):
    # Fast-converging preconditioned GMRES puts most of A P^{-1} v_j in the
    # current Krylov space; a Gram-Schmidt step that loses orthogonality there
    # stalls the residual estimate, which shows as extra iterations.
    alpha, dt = 1.5, 1.0 / 512
    h = 1.0 / (n + 1)
    xg = h * np.arange(1, n + 1)
    dp, dm = 1 + xg ** 2, 1 + (1 - xg) ** 2
    b = np.random.default_rng(0).uniform(-1, 1, n)
    prob = oracle.Problem1D(alpha=alpha, n=n, c0=h ** alpha / dt, dp=dp, dm=dm)
    ref = oracle.gmres(prob.matvec, b, Pinv=oracle.Tau1D.for_problem(prob).apply_inverse, restart=30, tol=tol,
                       maxiter=600)
    plan = fde.Plan(1, n, alpha, dt, dp=dp, dm=dm, method="gmres", restart=30, precision="f64")
    info = plan.solve(to_dev(gpu, b, "f64"), tol=tol, max_iters=600)
    assert info["status"] == fde.OK, info
    assert abs(info["iterations"] - ref.iterations) <= 1, (info["iterations"], ref.iterations)
    assert rel_err(info["x"].cpu().numpy(), ref.x) < 1e3 * tol


@pytest.mark.parametrize("alpha", [1.2, 1.5, 1.8])
def test_gmres_refinement_fp32_inner(gpu, alpha):
    """FP32 inner GMRES, FP64 outer residual and update: every solve reaches
    the FP64 tolerance and the refined solution matches the tight oracle."""
    n = 4095
    w = workloads.var_1d_time_stepping(n=n, alphas=(alpha,))[0]
    prob = oracle_problem_1d(w)
    b = prob.c0 * w["u0"]
    P = oracle.Tau1D.for_problem(prob)
    tight = oracle.gmres(prob.matvec, b, Pinv=P.apply_inverse, restart=30, tol=1e-12, maxiter=3000,
                         stop_on_estimate=True)
    plan = fde.Plan.from_workload(w, precision="f32_ir")
    info = plan.solve(to_dev(gpu, b, "f64"), tol=1e-8, inner_tol=1e-3, max_iters=20000, max_outer=200)
    x = info["x"].cpu().numpy()
    assert info["status"] == fde.OK, info
    assert np.linalg.norm(b - prob.matvec(x)) / np.linalg.norm(b) <= 1.01e-8 and info["relres"] <= 1e-8
    info2 = plan.solve(to_dev(gpu, b, "f64"), tol=1e-12, inner_tol=1e-3, max_iters=20000, max_outer=400)
    assert rel_err(info2["x"].cpu().numpy(), tight.x) < 1e-8


@pytest.mark.parametrize("case", ["1d", "2d"])
def test_pure_fp32_inner_solve(gpu, case):
    """The pure FP32 solve (no refinement) on the constant-coefficient PCG
    problems, asked for 1e-7: the FP64-checked relative residual is below 2e-6
    (FP32's attainable floor here is ~1.4e-6: the recurrence residual drifts
    from the true one by ~kappa u32) and the solution matches the tight FP64
    oracle to 1e-5."""
    if case == "1d":
        w = workloads.const_1d(n=1023)
        prob = oracle_problem_1d(w)
        P = oracle.Tau1D.for_problem(prob, shift=True)
    else:
        w = workloads.const_2d(n=127)
        h = 1.0 / 128
        prob = oracle.Problem2D(alpha=w["alpha"], beta=w["beta"], n1=127, n2=127, c0=h ** w["alpha"] / w["dt"],
                                sr=h ** w["alpha"] / h ** w["beta"], dp=w["dp"], dm=w["dm"], ep=w["ep"],
                                em=w["em"], scheme="wsgd2")
        P = oracle.Tau2D.for_problem(prob, shift=True)
    b = prob.c0 * w["b"]
    tight = oracle.pcg(prob.matvec, b, Pinv=P.apply_inverse, tol=1e-13, maxiter=500)
    plan = fde.Plan.from_workload(w, precision="f32")
    info = plan.solve(to_dev(gpu, b, "f64"), tol=1e-7)
    x = info["x"].cpu().numpy()
    relres = np.linalg.norm(b - prob.matvec(x)) / np.linalg.norm(b)
    assert relres <= 2e-6, (relres, info)
    assert abs(info["relres"] - relres) <= 1e-2 * relres
    assert rel_err(x, tight.x) < 1e-5


@pytest.mark.parametrize("n", [63, 255])
def test_gmres_left_paper_mode_example1(gpu, n):
    """Sec. 4 convention: left preconditioning, GMRES(20), x0 = 0, tol 1e-7."""
    from oracle.examples import example1_problem, example1_source, example1_exact
    prob, meta = example1_problem(1.5, n)
    x = meta["x"]
    plan = fde.Plan(1, n, 1.5, meta["ht"], len1=2.0, dp=prob.dp, dm=prob.dm, restart=20)
    P = oracle.Tau1D.for_problem(prob)
    u = example1_exact(x, 0.0)
    for m in range(1, 4):
        b = prob.c0 * u + meta["h"] ** 1.5 * example1_source(1.5, x, m * meta["ht"])
        ref = oracle.gmres(prob.matvec, b, Pinv=P.apply_inverse, side="left", restart=20, tol=1e-7)
        info = plan.solve(to_dev(gpu, b, "f64"), tol=1e-7, side="left")
        assert abs(info["iterations"] - ref.iterations) <= 1, (m, info, ref.iterations)
        assert rel_err(info["x"].cpu().numpy(), ref.x) < 1e-6
        u = ref.x


def test_batched_case1_instances(gpu):
    ws = workloads.const_1d_batch(count=24, kmin=8, kmax=11)
    plans, bs, xs, refs = [], [], [], []
    for w in ws:
        prob = oracle_problem_1d(w)
        b = prob.c0 * w["b"]
        P = oracle.Tau1D.for_problem(prob, shift=True)
        refs.append((prob, b, oracle.pcg(prob.matvec, b, Pinv=P.apply_inverse, tol=1e-8)))
        plans.append(fde.Plan.from_workload(w, precision="f32_ir"))
        bs.append(to_dev(gpu, b, "f64"))
        xs.append(gpu.zeros_like(bs[-1]))
    infos = fde.solve_batch(plans, bs, xs, tol=1e-8, inner_tol=1e-5)
    for (prob, b, ref), info, x in zip(refs, infos, xs):
        assert info["status"] == fde.OK, info
        xx = x.cpu().numpy()
        assert np.linalg.norm(b - prob.matvec(xx)) / np.linalg.norm(b) <= 1.01e-8
        assert rel_err(xx, ref.x) < 1e-6


def test_reassemble_all_on_side_streams_matches_one_by_one(gpu):
    """Plans reassembled on side streams at once give the same symbol data as
    one after another: the batch's solves after each are bit-identical, and
    the first instance matches the oracle."""
    from paper_1912_13304_gb300.solver import reassemble_all
    ws = workloads.const_1d_batch(count=20, kmin=8, kmax=12)
    plans = [fde.Plan.from_workload(w) for w in ws]
    bs = [p.c0 * to_dev(gpu, w["b"], "f64") for p, w in zip(plans, ws)]
    for p in plans:
        p.reassemble()
    xs1 = [gpu.zeros_like(b) for b in bs]
    inf1 = fde.solve_batch(plans, bs, xs1, tol=1e-10)
    reassemble_all(plans, streams=8)
    xs2 = [gpu.zeros_like(b) for b in bs]
    inf2 = fde.solve_batch(plans, bs, xs2, tol=1e-10)
    for a, b_, x1, x2 in zip(inf1, inf2, xs1, xs2):
        assert a["status"] == fde.OK and a["iterations"] == b_["iterations"], (a, b_)
        assert gpu.equal(x1, x2)
    prob = oracle_problem_1d(ws[0])
    b0 = prob.c0 * ws[0]["b"]
    ref = oracle.pcg(prob.matvec, b0, Pinv=oracle.Tau1D.for_problem(prob, shift=True).apply_inverse, tol=1e-13)
    assert rel_err(xs2[0].cpu().numpy(), ref.x) < 1e-8


@pytest.mark.parametrize("precision", ["f64", "f32_ir"])
@pytest.mark.parametrize("n", [63, 255])
def test_2d_pcg_shifted(gpu, n, precision):
    w = workloads.const_2d(n=n)
    h = 1.0 / (n + 1)
    prob = oracle.Problem2D(alpha=w["alpha"], beta=w["beta"], n1=n, n2=n, c0=h ** w["alpha"] / w["dt"],
                            sr=h ** w["alpha"] / h ** w["beta"], dp=w["dp"], dm=w["dm"], ep=w["ep"], em=w["em"],
                            scheme="wsgd2")
    b = prob.c0 * w["b"]
    P = oracle.Tau2D.for_problem(prob, shift=True)
    ref = oracle.pcg(prob.matvec, b, Pinv=P.apply_inverse, tol=1e-8)
    plan = fde.Plan.from_workload(w, precision=precision)
    info = plan.solve(to_dev(gpu, b, "f64"), tol=1e-8, inner_tol=1e-5)
    assert info["status"] == fde.OK, info
    if precision == "f64":
        assert abs(info["iterations"] - ref.iterations) <= 1, (info, ref.iterations)
    x = info["x"].cpu().numpy()
    assert np.linalg.norm(b - prob.matvec(x)) / np.linalg.norm(b) <= 1.01e-8
    assert rel_err(x, ref.x) < 1e-6


@pytest.mark.parametrize("n", [31, 127])
def test_2d_gmres_variable(gpu, n):
    w = workloads.var_2d_time_stepping(n=n)
    h = 1.0 / (n + 1)
    prob = oracle.Problem2D(alpha=w["alpha"], beta=w["beta"], n1=n, n2=n, c0=h ** w["alpha"] / w["dt"],
                            sr=h ** w["alpha"] / h ** w["beta"], dp=w["dp"], dm=w["dm"], ep=w["ep"], em=w["em"],
                            scheme="wsgd2")
    b = prob.c0 * w["u0"]
    P = oracle.Tau2D.for_problem(prob)
    ref = oracle.gmres(prob.matvec, b, Pinv=P.apply_inverse, x0=w["u0"], restart=20, tol=1e-8)
    plan = fde.Plan.from_workload(w)
    info = plan.solve(to_dev(gpu, b, "f64"), x=to_dev(gpu, w["u0"], "f64"), tol=1e-8)
    assert info["status"] == fde.OK, info
    assert abs(info["iterations"] - ref.iterations) <= 1, (info, ref.iterations)
    x = info["x"].cpu().numpy()
    assert np.linalg.norm(b - prob.matvec(x)) / np.linalg.norm(b) <= 1.01e-8


def test_zero_rhs_and_iteration_cap(gpu):
    n = 255
    plan, prob = make_1d(gpu, n, "var")
    z = gpu.zeros(n, dtype=gpu.float64, device="cuda")
    info = plan.solve(z, x=gpu.ones(n, dtype=gpu.float64, device="cuda"))
    assert info["status"] == fde.OK and float(info["x"].abs().max()) == 0.0
    b = to_dev(gpu, np.random.default_rng(0).uniform(-1, 1, n), "f64")
    info = plan.solve(b, max_iters=2, tol=1e-12)
    assert info["status"] == fde.ENOCONV and info["iterations"] == 2
    assert 0 < info["relres"] < 1


def test_full_size_variable_coefficient_step(gpu):
    """One implicit-Euler step of the n = 65535 workload (alpha = 1.8) on the
    split-line path: device relres re-checked by the oracle's direct sums.
    At kappa(M) ~ 1e7 both residual evaluations carry rounding of order
    u ||M|| ||x|| / ||b|| ~ 1e-9, so they agree to that level, not to 1e-3."""
    w = workloads.var_1d_time_stepping(alphas=(1.8,))[0]
    prob = oracle_problem_1d(w)
    b = prob.c0 * w["u0"]
    plan = fde.Plan.from_workload(w)
    info = plan.solve(to_dev(gpu, b, "f64"), x=to_dev(gpu, w["u0"], "f64"), tol=1e-8)
    assert info["status"] == fde.OK, info
    x = info["x"].cpu().numpy()
    rr = np.linalg.norm(b - prob.matvec(x, "direct")) / np.linalg.norm(b)
    assert rr <= 1.01e-8 and abs(rr - info["relres"]) <= 2e-9
    assert info["iterations"] <= 25


def test_batched_balanced_teams_match_even_split(gpu):
    # Team sizes from the previous solve's iteration counts change only the
    # reduction order: the same iterations (+-1) and the same solutions.
    import torch
    ws = workloads.var_1d_time_stepping(n=16383, alphas=(1.2, 1.5, 1.8))
    plans = [fde.Plan.from_workload(w) for w in ws]
    bs = [plans[i].rhs(to_dev(gpu, w["u0"], "f64")) for i, w in enumerate(ws)]
    xs0 = [to_dev(gpu, w["u0"], "f64") for w in ws]
    info = torch.zeros(len(ws) * fde.INFO_BYTES, dtype=torch.uint8, device="cuda")
    # tol 1e-8: at n = 16383, alpha = 1.8 an FP64 evaluation of the residual is
    # itself uncertain near 1e-10 (||D T x|| / ||b|| ~ 1e6)
    even = fde.solve_batch(plans, bs, xs0, tol=1e-8, max_iters=3000, info_dev=info)
    its = [i["iterations"] for i in even]
    assert len(set(its)) > 1, its           # unequal work, so the split is uneven
    xs1 = [to_dev(gpu, w["u0"], "f64") for w in ws]
    bal = fde.solve_batch(plans, bs, xs1, tol=1e-8, max_iters=3000, info_dev=info, balance=True)
    # Both solutions satisfy relres <= 1e-8, so they may differ by up to
    # kappa(M) * 1e-8 (kappa ~ 1e6 at n = 16383, alpha = 1.8); each is checked
    # against the oracle's residual instead.
    for e, b_, x0, x1, w, p in zip(even, bal, xs0, xs1, ws, plans):
        assert e["status"] == fde.OK and b_["status"] == fde.OK, (e, b_)
        assert abs(b_["iterations"] - e["iterations"]) <= 1, (e["iterations"], b_["iterations"])
        prob = oracle_problem_1d(w)
        bb = prob.c0 * w["u0"]
        for x in (x0, x1):
            rr = np.linalg.norm(bb - prob.matvec(x.cpu().numpy())) / np.linalg.norm(bb)
            assert rr <= 1.01e-8, (rr, e, b_)
        assert rel_err(x1.cpu().numpy(), x0.cpu().numpy()) < 1e-2


def test_graph_time_stepping_replays_the_eager_steps(gpu):
    # The captured loop launches the same kernels on the same data: the
    # replayed steps reproduce the eager ones bit for bit (deterministic
    # reductions), and every replayed step reports convergence.
    import torch
    from paper_1912_13304_gb300.solver import TimeStepper
    ws = workloads.var_1d_time_stepping(n=16383, alphas=(1.2, 1.8), steps=3)
    plans = [fde.Plan.from_workload(w) for w in ws]
    u0 = [to_dev(gpu, w["u0"], "f64") for w in ws]
    ue = [x.clone() for x in u0]
    eager = TimeStepper(plans, ue, 3, tol=1e-8, max_iters=3000, graph=False)
    eager.run()
    ug = [x.clone() for x in u0]
    graph = TimeStepper(plans, ug, 3, tol=1e-8, max_iters=3000, graph=True)
    for _ in range(2):                     # replay twice from the same start
        for x, x0 in zip(ug, u0):
            x.copy_(x0)
        graph.run()
        torch.cuda.synchronize()
        for a, b in zip(ug, ue):
            assert torch.equal(a, b)
        assert graph.infos() == eager.infos()
    # every replayed step converged (the device's FP64 true residual); the
    # eager path is checked against the oracle by the step tests above
    for step in graph.infos():
        for inf in step:
            assert inf["status"] == fde.OK and inf["relres"] <= 1e-8, inf


@pytest.mark.parametrize("precision", ["f64", "f32_ir"])
def test_batched_256_instances_full_size(gpu, precision):
    # The full batched workload (n up to 16383, so one-CTA teams also run the
    # split-line layout): every instance converges, and a sample spanning the
    # sizes matches the oracle's PCG iteration counts and residuals.
    ws = workloads.const_1d_batch()
    plans = [fde.Plan.from_workload(w, precision=precision) for w in ws]
    bs = [to_dev(gpu, p.c0 * w["b"], "f64") for p, w in zip(plans, ws)]
    xs = [gpu.zeros_like(b) for b in bs]
    infos = fde.solve_batch(plans, bs, xs, tol=1e-8, max_iters=2000, inner_tol=1e-4, max_outer=100)
    for inf in infos:
        assert inf["status"] == fde.OK and inf["relres"] <= 1e-8, inf
    sizes = sorted(range(len(ws)), key=lambda i: ws[i]["n1"])
    sample = sorted(set(sizes[::40] + [sizes[-1], sizes[-2]]))
    for i in sample:
        w = ws[i]
        prob = oracle_problem_1d(w)
        b = prob.c0 * w["b"]
        ref = oracle.pcg(prob.matvec, b, Pinv=oracle.Tau1D.for_problem(prob, shift=True).apply_inverse, tol=1e-8)
        if precision == "f64":
            assert abs(infos[i]["iterations"] - ref.iterations) <= 1, (w["n1"], infos[i], ref.iterations)
        x = xs[i].cpu().numpy()
        assert np.linalg.norm(b - prob.matvec(x)) / np.linalg.norm(b) <= 1.01e-8, (w["n1"], infos[i])


def test_autotuned_schedule_solves_match_oracle(gpu):
    n = 16383
    w = workloads.var_1d_time_stepping(n=n, alphas=(1.5,))[0]
    prob = oracle_problem_1d(w)
    b = prob.c0 * w["u0"]
    ref = oracle.gmres(prob.matvec, b, Pinv=oracle.Tau1D.for_problem(prob).apply_inverse, x0=w["u0"], restart=30,
                       tol=1e-8)
    plan = fde.Plan.from_workload(w)
    ctas, lp1 = plan.autotune()
    info = plan.solve(to_dev(gpu, b, "f64"), x=to_dev(gpu, w["u0"], "f64"), tol=1e-8)
    assert info["status"] == fde.OK, (info, ctas, lp1)
    assert abs(info["iterations"] - ref.iterations) <= 1, (info["iterations"], ref.iterations, ctas, lp1)
    x = info["x"].cpu().numpy()
    assert np.linalg.norm(b - prob.matvec(x)) / np.linalg.norm(b) <= 1.01e-8
    # a second plan of the same shape takes the cached choice
    plan2 = fde.Plan.from_workload(w)
    assert plan2.autotune() == (ctas, lp1)


def test_autotuned_schedule_full_size_and_2d(gpu):
    # n = 65535: the tuned schedule against the default one (same iterations)
    w = workloads.var_1d_time_stepping(alphas=(1.8,))[0]
    infos = []
    for tune in (False, True):
        plan = fde.Plan.from_workload(w)
        if tune:
            plan.autotune()
        b = plan.rhs(to_dev(gpu, w["u0"], "f64"))
        infos.append(plan.solve(b, x=to_dev(gpu, w["u0"], "f64"), tol=1e-8))
    assert all(i["status"] == fde.OK and i["relres"] <= 1e-8 for i in infos), infos
    assert abs(infos[0]["iterations"] - infos[1]["iterations"]) <= 1
    # 2D: team size only
    w2 = workloads.var_2d_time_stepping(n=255, steps=1)
    plan = fde.Plan.from_workload(w2, precision="f32_ir")
    ctas, lp1 = plan.autotune()
    assert lp1 == 0 and ctas >= 16
    h = 1.0 / 256
    prob = oracle.Problem2D(alpha=w2["alpha"], beta=w2["beta"], n1=255, n2=255, c0=h ** w2["alpha"] / w2["dt"],
                            sr=h ** w2["alpha"] / h ** w2["beta"], dp=w2["dp"], dm=w2["dm"], ep=w2["ep"],
                            em=w2["em"], scheme="wsgd2")
    b = prob.c0 * w2["u0"]
    info = plan.solve(to_dev(gpu, b, "f64"), x=to_dev(gpu, w2["u0"], "f64"), tol=1e-8, inner_tol=1e-4)
    assert info["status"] == fde.OK, info
    x = info["x"].cpu().numpy()
    assert np.linalg.norm(b - prob.matvec(x)) / np.linalg.norm(b) <= 1.01e-8


@pytest.mark.parametrize("dim", [1, 2])
def test_step_rhs_crank_nicolson(gpu, dim):
    # b = (2 c0 I - M) u + 2 h^alpha f (Sec. 1.4) against the oracle's matvec
    rng = np.random.default_rng(21 + dim)
    if dim == 1:
        n, alpha, dt = 1023, 1.6, 1.0 / 64
        h = 1.0 / (n + 1)
        xg = h * np.arange(1, n + 1)
        dp, dm = 1 + xg, 2 - xg
        plan = fde.Plan(1, n, alpha, dt, scheme="cn", dp=dp, dm=dm)
        prob = oracle.Problem1D(alpha=alpha, n=n, c0=2 * h ** alpha / dt, dp=dp, dm=dm)
        N, ha = n, h ** alpha
    else:
        from oracle.examples import example2_problem
        prob, meta = example2_problem(1.4, 1.7, 63)
        plan = fde.Plan(2, 63, 1.4, meta["ht"], n2=63, beta=1.7, len1=2.0, len2=2.0, scheme="cn", weights="wsgd2",
                        dp=prob.dp, dm=prob.dm, ep=prob.ep, em=prob.em)
        N, ha = 63 * 63, meta["h"] ** 1.4
    u = rng.uniform(-1, 1, N)
    f = rng.uniform(-1, 1, N)
    b = plan.rhs(to_dev(gpu, u, "f64"), f=to_dev(gpu, f, "f64")).cpu().numpy()
    assert abs(plan.c0 - prob.c0) <= 1e-14 * prob.c0
    ref = 2 * prob.c0 * u - prob.matvec(u) + 2 * ha * f
    scale = np.max(np.abs(2 * prob.c0 * u)) + np.max(np.abs(prob.matvec(u)))
    assert np.max(np.abs(b - ref)) / scale < 1e-12


def test_crank_nicolson_example2_march_matches_oracle(gpu):
    # Example 2 (Sec. 4.2): the whole Crank-Nicolson march in paper mode (left
    # GMRES(20), tol 1e-7, tau(F) D), right-hand sides built on the device
    from oracle.examples import example2_exact, example2_march, example2_problem, example2_source
    alpha, beta, n = 1.5, 1.5, 31          # n + 1 = 2^k (the library's grids); 31 steps
    u_ref, its_ref, exact = example2_march(alpha, beta, n)
    prob, meta = example2_problem(alpha, beta, n)
    X, Y, h, ht = meta["X"], meta["Y"], meta["h"], meta["ht"]
    plan = fde.Plan(2, n, alpha, ht, n2=n, beta=beta, len1=2.0, len2=2.0, scheme="cn", weights="wsgd2",
                    dp=prob.dp, dm=prob.dm, ep=prob.ep, em=prob.em, restart=20)
    u = to_dev(gpu, example2_exact(X, Y, 0.0).reshape(-1), "f64")
    its = []
    for m in range(1, meta["steps"] + 1):
        f = to_dev(gpu, example2_source(alpha, beta, X, Y, (m - 0.5) * ht).reshape(-1), "f64")
        b = plan.rhs(u, f=f)
        info = plan.solve(b, tol=1e-7, side="left")
        assert info["status"] == fde.OK, (m, info)
        u = info["x"]
        its.append(info["iterations"])
    assert all(abs(a - r) <= 1 for a, r in zip(its, its_ref)), (its, its_ref)
    ug = u.cpu().numpy()
    assert rel_err(ug, u_ref) < 1e-6
    # and the discretisation error is the oracle's (the paper's O(h^2) scheme)
    assert abs(np.max(np.abs(ug - exact)) - np.max(np.abs(u_ref - exact))) < 1e-6 * np.max(np.abs(exact))


@pytest.mark.parametrize("n", [63, 255])
def test_gmres_left_ftilde_example1(gpu, n):
    """P_F-tilde (Sec. 4, Table 2) in paper mode on Example 1."""
    from oracle.examples import example1_exact, example1_problem, example1_source
    prob, meta = example1_problem(1.5, n)
    x = meta["x"]
    plan = fde.Plan(1, n, 1.5, meta["ht"], len1=2.0, dp=prob.dp, dm=prob.dm, restart=20, order="tau_df")
    P = oracle.Tau1D.for_problem(prob, order="tau_df")
    u = example1_exact(x, 0.0)
    for m in range(1, 4):
        b = prob.c0 * u + meta["h"] ** 1.5 * example1_source(1.5, x, m * meta["ht"])
        ref = oracle.gmres(prob.matvec, b, Pinv=P.apply_inverse, side="left", restart=20, tol=1e-7)
        info = plan.solve(to_dev(gpu, b, "f64"), tol=1e-7, side="left")
        assert abs(info["iterations"] - ref.iterations) <= 1, (m, info, ref.iterations)
        assert rel_err(info["x"].cpu().numpy(), ref.x) < 1e-6
        u = ref.x


@pytest.mark.parametrize("alpha", [1.2, 1.8])
def test_refinement_switches_to_fp64_when_fp32_corrections_stall(gpu, alpha):
    # alpha = 1.8 at n = 16383: kappa(M) u32 log2 L > 1, the FP32 corrections
    # barely shrink the residual and the solve finishes in FP64 (close to the
    # FP64 iteration count; FP32 refinement alone needed hundreds more).
    # alpha = 1.2: the FP32 corrections contract and refinement continues.
    n = 16383
    w = workloads.var_1d_time_stepping(n=n, alphas=(alpha,))[0]
    prob = oracle_problem_1d(w)
    b = prob.c0 * w["u0"]
    i64 = fde.Plan.from_workload(w).solve(to_dev(gpu, b, "f64"), x=to_dev(gpu, w["u0"], "f64"), tol=1e-8)
    pir = fde.Plan.from_workload(w, precision="f32_ir")
    iir = pir.solve(to_dev(gpu, b, "f64"), x=to_dev(gpu, w["u0"], "f64"), tol=1e-8, inner_tol=1e-3,
                    max_iters=20000, max_outer=200)
    assert iir["status"] == fde.OK and iir["relres"] <= 1e-8, iir
    x = iir["x"].cpu().numpy()
    assert np.linalg.norm(b - prob.matvec(x)) / np.linalg.norm(b) <= 1.01e-8
    if alpha == 1.8:
        assert iir["iterations"] <= i64["iterations"] + 150, (iir, i64)
    else:
        assert iir["outer"] >= 2, iir


@pytest.mark.parametrize("n", [63, 255])
def test_gmres_left_tridiagonal_example1(gpu, n):
    """P_tri (Sec. 4, Table 2) in paper mode on Example 1: left GMRES(20),
    x0 = 0, tol 1e-7, iterations within +-1 of the oracle's per step."""
    from oracle.examples import example1_exact, example1_problem, example1_source
    prob, meta = example1_problem(1.5, n)
    x = meta["x"]
    plan = fde.Plan(1, n, 1.5, meta["ht"], len1=2.0, dp=prob.dp, dm=prob.dm, restart=20, order="tri")
    P = oracle.Tri1D.for_problem(prob)
    u = example1_exact(x, 0.0)
    for m in range(1, 4):
        b = prob.c0 * u + meta["h"] ** 1.5 * example1_source(1.5, x, m * meta["ht"])
        ref = oracle.gmres(prob.matvec, b, Pinv=P.apply_inverse, side="left", restart=20, tol=1e-7)
        info = plan.solve(to_dev(gpu, b, "f64"), tol=1e-7, side="left")
        assert abs(info["iterations"] - ref.iterations) <= 1, (m, info, ref.iterations)
        assert rel_err(info["x"].cpu().numpy(), ref.x) < 1e-6
        u = ref.x


@pytest.mark.parametrize("precision", ["f64", "f32_ir"])
@pytest.mark.parametrize("n", [1023, 16383])
def test_gmres_right_tridiagonal_variable_coefficients(gpu, n, precision):
    # right-preconditioned GMRES(30) with P_tri on the variable-coefficient
    # step (alpha = 1.2, where P_tri is competitive), both line layouts
    w = workloads.var_1d_time_stepping(n=n, alphas=(1.2,))[0]
    prob = oracle_problem_1d(w)
    b = prob.c0 * w["u0"]
    ref = oracle.gmres(prob.matvec, b, Pinv=oracle.Tri1D.for_problem(prob).apply_inverse, x0=w["u0"],
                       restart=30, tol=1e-8, maxiter=3000)
    plan = fde.Plan.from_workload(w, order="tri", precision=precision)
    info = plan.solve(to_dev(gpu, b, "f64"), x=to_dev(gpu, w["u0"], "f64"), tol=1e-8, max_iters=3000,
                      inner_tol=1e-4, max_outer=100)
    assert info["status"] == fde.OK, info
    if precision == "f64":
        assert abs(info["iterations"] - ref.iterations) <= 1, (info["iterations"], ref.iterations)
    x = info["x"].cpu().numpy()
    assert np.linalg.norm(b - prob.matvec(x)) / np.linalg.norm(b) <= 1.01e-8
