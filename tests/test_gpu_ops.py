"""Parity of the CUDA operators (through the C ABI) with the CPU oracle.

y = M x (fde_toeplitz_matvec) and z = P^{-1} r (fde_tau_solve), element by
element, for 1D lines held by one CTA and lines split across CTAs, 2D planes,
both precisions and every preconditioner variant.

Tolerances (max-norm error relative to max |reference|): C u log2(L) per
operator and precision, u the unit roundoff and L the transform length (see
TOL_C below for the constants and how they were set).
"""

import numpy as np
import pytest

import oracle
import paper_1912_13304_gb300 as fde

pytestmark = pytest.mark.gpu

# Bound on the relative max-norm error of an operator application whose
# transforms have L real points per line: C u log2(L), u the unit roundoff.
# An L-point FFT's rounding error grows like u log2 L relative to the largest
# entry; for the tau solve the division by the symbol samples amplifies the
# transform errors and the signal alike (both sit in the smoothest sine
# modes), so the relative error keeps that form.  The constants are about
# four to eight times the largest ratio err / (u log2 L) measured on a GB300
# over every size and variant below (FP32: 0.6 for the matvec, 1.3 for tau;
# FP64 matvec: 3.7, where the dense FP64 reference itself carries that).  The
# FP64 tau bound grows with L beyond 8192: its reference, the oracle's symbol
# from the complex power (1 - e^{i theta})^alpha, loses relative accuracy
# like 1/theta_1 ~ L at the smallest sample, which the tau solve weighs most
# (measured ratios 77, 178, 461 at L = 2^14, 2^15, 2^17).
UNIT = {"f64": 2.0 ** -53, "f32": 2.0 ** -24}
TOL_C = {("mv", "f64"): 16.0, ("tau", "f64"): 64.0, ("mv", "f32"): 6.0, ("tau", "f32"): 10.0}


def tol(op, dtype, L):
    """Bound on the relative max-norm error of one operator application whose
    transforms have L real points per line."""
    c = TOL_C[(op, dtype)]
    if (op, dtype) == ("tau", "f64"):
        c = max(c, L / 64.0)
    return c * UNIT[dtype] * max(np.log2(L), 1.0)


def L1(n):
    return 2 * (n + 1)


def rel_err(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def coeffs_1d(kind, n):
    h = 1.0 / (n + 1)
    x = h * np.arange(1, n + 1)
    if kind == "var":
        return 1 + x ** 2, 1 + (1 - x) ** 2
    if kind == "sym":
        d = 1 + np.sin(3 * x) ** 2
        return d, d
    return np.full(n, 1.3), np.full(n, 1.3)


def make_1d(gpu, n, kind, alpha=1.5, dt=1 / 512, weights="gl1", shift=False, order="tau_d", precision="f64"):
    dp, dm = coeffs_1d(kind, n)
    h = 1.0 / (n + 1)
    if kind == "const":
        plan = fde.Plan(1, n, alpha, dt, dp_const=dp[0], dm_const=dm[0], weights=weights, tau_shift=shift,
                        order=order, precision=precision)
    else:
        plan = fde.Plan(1, n, alpha, dt, dp=dp, dm=dm if kind == "var" else dp, weights=weights, tau_shift=shift,
                        order=order, precision=precision)
    prob = oracle.Problem1D(alpha=alpha, n=n, c0=h ** alpha / dt, dp=dp, dm=dm, scheme=weights)
    return plan, prob


def to_dev(gpu, v, dtype):
    return gpu.tensor(np.asarray(v), dtype=gpu.float64 if dtype == "f64" else gpu.float32, device="cuda")


SIZES_1D = [1, 3, 7, 63, 1023, 4095, 8191, 16383]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("kind", ["var", "sym", "const"])
@pytest.mark.parametrize("n", SIZES_1D)
def test_matvec_1d(gpu, n, kind, dtype):
    plan, prob = make_1d(gpu, n, kind)
    x = np.random.default_rng(n).uniform(-1, 1, n)
    y = plan.matvec(to_dev(gpu, x, dtype)).double().cpu().numpy()
    ref = prob.matvec(x, "direct" if n > 4096 else "dense")
    assert rel_err(y, ref) < tol("mv", dtype, L1(n))


@pytest.mark.parametrize("weights", ["gl1", "wsgd2"])
@pytest.mark.parametrize("alpha", [1.1, 1.9])
def test_matvec_1d_weights_and_orders(gpu, weights, alpha):
    n = 511
    plan, prob = make_1d(gpu, n, "var", alpha=alpha, weights=weights)
    x = np.random.default_rng(3).uniform(-1, 1, n)
    y = plan.matvec(to_dev(gpu, x, "f64")).cpu().numpy()
    assert rel_err(y, prob.matvec(x)) < tol("mv", "f64", L1(n))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("variant", ["tau_d", "d_tau", "shift"])
@pytest.mark.parametrize("n", SIZES_1D)
def test_tau_1d(gpu, n, variant, dtype):
    kind = "const" if variant == "shift" else "var"
    plan, prob = make_1d(gpu, n, kind, shift=variant == "shift", order="d_tau" if variant == "d_tau" else "tau_d")
    P = oracle.Tau1D.for_problem(prob, shift=variant == "shift", order="d_tau" if variant == "d_tau" else "tau_d")
    r = np.random.default_rng(n + 1).uniform(-1, 1, n)
    z = plan.tau(to_dev(gpu, r, dtype)).double().cpu().numpy()
    assert rel_err(z, P.apply_inverse(r)) < tol("tau", dtype, L1(n))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n", [1, 7, 63, 1023, 4095, 16383, 65535])
def test_tau_1d_ftilde(gpu, n, dtype):
    # P_F-tilde (Table 2): D_j folded into the symbol samples
    plan, prob = make_1d(gpu, n, "var", order="tau_df")
    P = oracle.Tau1D.for_problem(prob, order="tau_df")
    r = np.random.default_rng(n + 9).uniform(-1, 1, n)
    z = plan.tau(to_dev(gpu, r, dtype)).double().cpu().numpy()
    assert rel_err(z, P.apply_inverse(r)) < tol("tau", dtype, L1(n))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("order", ["tau_d", "d_tau"])
@pytest.mark.parametrize("n", [7, 1023, 4095, 16383, 65535])
def test_tau_1d_shifted_variable_coefficients(gpu, n, order, dtype):
    # the shift c0/mean(D) beside a variable D (assembled on the device: the
    # mean is a device reduction), every line layout
    plan, prob = make_1d(gpu, n, "var", shift=True, order=order)
    P = oracle.Tau1D.for_problem(prob, shift=True, order=order)
    r = np.random.default_rng(n + 5).uniform(-1, 1, n)
    z = plan.tau(to_dev(gpu, r, dtype)).double().cpu().numpy()
    assert rel_err(z, P.apply_inverse(r)) < tol("tau", dtype, L1(n))


# P_tri by parallel cyclic reduction against the oracle's Thomas algorithm:
# both are Gaussian elimination on a strictly diagonally dominant tridiagonal
# matrix (error a few ulps times log2 n relative to the solution)
TRI_TOL = {"f64": 1e-12, "f32": 2e-5}


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("alpha", [1.1, 1.9])
@pytest.mark.parametrize("n", [1, 2 ** 2 - 1, 63, 1023, 4095, 8191, 65535])
def test_tri_1d(gpu, n, alpha, dtype):
    # every line layout: one CTA's shared memory up to n = 4095, the team's
    # global-memory rounds beyond
    plan, prob = make_1d(gpu, n, "var", alpha=alpha, order="tri")
    P = oracle.Tri1D.for_problem(prob)
    r = np.random.default_rng(n + 17).uniform(-1, 1, n)
    z = plan.tau(to_dev(gpu, r, dtype)).double().cpu().numpy()
    assert rel_err(z, P.apply_inverse(r)) < TRI_TOL[dtype]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_full_size_1d_line_split_across_ctas(gpu, dtype):
    """n = 65535 (the variable-coefficient workload): sampled rows of M x by
    their definition, and the whole tau solve."""
    n = 65535
    plan, prob = make_1d(gpu, n, "var", alpha=1.8)
    rng = np.random.default_rng(11)
    x = rng.uniform(-1, 1, n)
    y = plan.matvec(to_dev(gpu, x, dtype)).double().cpu().numpy()
    rows = np.concatenate([[0, 1, 2, n // 2, n - 2, n - 1], rng.integers(0, n, 40)])
    ref = prob.matvec_rows(x, rows)
    scale = np.max(np.abs(prob.matvec_rows(x, rng.integers(0, n, 200))))
    assert np.max(np.abs(y[rows] - ref)) / scale < tol("mv", dtype, L1(n))
    P = oracle.Tau1D.for_problem(prob)
    z = plan.tau(to_dev(gpu, x, dtype)).double().cpu().numpy()
    assert rel_err(z, P.apply_inverse(x)) < tol("tau", dtype, L1(n))


SIZES_2D = [(1, 1), (3, 7), (15, 31), (63, 63), (127, 255), (511, 127)]


def make_2d(gpu, n1, n2, kind, alpha=1.3, beta=1.8, dt=1 / 256, shift=False, order="tau_d", precision="f64"):
    h1, h2 = 1.0 / (n1 + 1), 1.0 / (n2 + 1)
    X, Y = np.meshgrid(h1 * np.arange(1, n1 + 1), h2 * np.arange(1, n2 + 1), indexing="xy")
    if kind == "var":
        dp, dm, ep, em = 1 + X + Y, 2 - X, 1 + X * Y, 1 + Y ** 2
    else:
        dp = dm = np.full((n2, n1), 1.2)
        ep = em = np.full((n2, n1), 0.8)
    if kind == "var":
        plan = fde.Plan(2, n1, alpha, dt, n2=n2, beta=beta, weights="wsgd2", dp=dp, dm=dm, ep=ep, em=em,
                        order=order, precision=precision)
    else:
        plan = fde.Plan(2, n1, alpha, dt, n2=n2, beta=beta, weights="wsgd2", dp_const=1.2, dm_const=1.2,
                        ep_const=0.8, em_const=0.8, tau_shift=shift, order=order, precision=precision)
    prob = oracle.Problem2D(alpha=alpha, beta=beta, n1=n1, n2=n2, c0=h1 ** alpha / dt,
                            sr=h1 ** alpha / h2 ** beta, dp=dp, dm=dm, ep=ep, em=em, scheme="wsgd2")
    return plan, prob


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("kind", ["var", "const"])
@pytest.mark.parametrize("n1,n2", SIZES_2D)
def test_matvec_2d(gpu, n1, n2, kind, dtype):
    plan, prob = make_2d(gpu, n1, n2, kind)
    x = np.random.default_rng(n1 * n2).uniform(-1, 1, n1 * n2)
    y = plan.matvec(to_dev(gpu, x, dtype)).double().cpu().numpy()
    assert rel_err(y, prob.matvec(x)) < tol("mv", dtype, 2 * (max(n1, n2) + 1))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("variant", ["tau_d", "d_tau", "shift"])
@pytest.mark.parametrize("n1,n2", SIZES_2D)
def test_tau_2d(gpu, n1, n2, variant, dtype):
    kind = "const" if variant == "shift" else "var"
    order = "d_tau" if variant == "d_tau" else "tau_d"
    plan, prob = make_2d(gpu, n1, n2, kind, shift=variant == "shift", order=order)
    P = oracle.Tau2D.for_problem(prob, shift=variant == "shift", order=order)
    r = np.random.default_rng(n1 + n2).uniform(-1, 1, n1 * n2)
    z = plan.tau(to_dev(gpu, r, dtype)).double().cpu().numpy()
    assert rel_err(z, P.apply_inverse(r)) < tol("tau", dtype, 2 * (max(n1, n2) + 1))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n", [2047, 4095])
def test_full_size_2d_plane(gpu, n, dtype):
    """2047^2 and 4095^2 variable coefficients (L = 4096 and 8192 per axis):
    sampled entries of M x by their row definition, the whole product against
    the oracle's FFT-convolution form, and the whole tau solve through the
    library DST-I."""
    import os
    plan, prob = make_2d(gpu, n, n, "var")
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, n * n)
    y = plan.matvec(to_dev(gpu, x, dtype)).double().cpu().numpy()
    rows = np.concatenate([[0, 0, n - 1, n - 1, n // 2], rng.integers(0, n, 30)])
    cols = np.concatenate([[0, n - 1, 0, n - 1, n // 3], rng.integers(0, n, 30)])
    ref = prob.matvec_entries(x, rows, cols)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(y.reshape(n, n)[rows, cols] - ref)) / scale < tol("mv", dtype, 2 * (n + 1))
    oracle.set_fft_workers(os.cpu_count() or 1)
    try:
        assert rel_err(y, prob.matvec(x, "fft")) < tol("mv", dtype, 2 * (n + 1))
        P = oracle.Tau2D.for_problem(prob)
        z = plan.tau(to_dev(gpu, x, dtype)).double().cpu().numpy()
        assert rel_err(z, P.apply_inverse(x)) < tol("tau", dtype, 2 * (n + 1))
    finally:
        oracle.set_fft_workers(1)


def test_step_rhs(gpu):
    n = 1023
    plan, prob = make_1d(gpu, n, "var")
    rng = np.random.default_rng(2)
    u, f = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    b = plan.rhs(to_dev(gpu, u, "f64"), to_dev(gpu, f, "f64")).cpu().numpy()
    h = 1.0 / (n + 1)
    ref = prob.c0 * u + h ** 1.5 * f
    assert rel_err(b, ref) < 1e-15


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n", [4095, 16383, 65535])
def test_every_split_schedule_1d(gpu, n, dtype):
    # every four-step factorisation n + 1 = P1 x P2 the shared memory admits,
    # with a small and the full team, gives the same operators
    plan, prob = make_1d(gpu, n, "var", alpha=1.7)
    P = oracle.Tau1D.for_problem(prob)
    rng = np.random.default_rng(n + 2)
    x = rng.uniform(-1, 1, n)
    rows = np.concatenate([[0, 1, n // 2, n - 1], rng.integers(0, n, 30)])
    ref_rows = prob.matvec_rows(x, rows)
    scale = np.max(np.abs(prob.matvec_rows(x, rng.integers(0, n, 100))))
    z_ref = P.apply_inverse(x)
    logn = int(np.log2(n + 1))
    tried = 0
    for lp1 in range(4, logn // 2 + 1):
        for ctas in (16, 0):
            try:
                plan.set_schedule(ctas, lp1)
            except fde.FdeError as e:
                assert e.status == fde.EINVAL
                continue
            tried += 1
            y = plan.matvec(to_dev(gpu, x, dtype)).double().cpu().numpy()
            assert np.max(np.abs(y[rows] - ref_rows)) / scale < tol("mv", dtype, L1(n)), (lp1, ctas)
            z = plan.tau(to_dev(gpu, x, dtype)).double().cpu().numpy()
            assert rel_err(z, z_ref) < tol("tau", dtype, L1(n)), (lp1, ctas)
    assert tried >= 2
    plan.set_schedule(0, 0)
    y = plan.matvec(to_dev(gpu, x, dtype)).double().cpu().numpy()
    assert np.max(np.abs(y[rows] - ref_rows)) / scale < tol("mv", dtype, L1(n))


def test_schedule_validation(gpu):
    plan, _ = make_1d(gpu, 1023, "var")
    for bad in ((-1, 0), (0, -1), (0, 3), (0, 6)):     # 2^6 > sqrt(1024): P1 > P2
        with pytest.raises(fde.FdeError):
            plan.set_schedule(*bad)
    plan2, _ = make_2d(gpu, 63, 63, "var")
    with pytest.raises(fde.FdeError):
        plan2.set_schedule(0, 4)
    plan2.set_schedule(16, 0)
