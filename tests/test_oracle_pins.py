"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: library
routines (binomials, LAPACK, the DST-I), closed forms, textbook identities,
numerical quadrature of the symbols, and the values printed in Tables 1-4.
"""

import math

import numpy as np
import pytest
import scipy.special

import oracle
from oracle import (GL1, WSGD2, ORDER_D_TAU, ORDER_TAU_D, Problem1D, Problem2D, Tau1D,
                    Tau2D, gmres, grunwald_weights, pcg, preconditioned_condition_number,
                    sine_matrix, symbol_g, symbol_p, symbol_q, symbol_w, tau_grid,
                    toeplitz_from_weights, wsgd_weights)
from oracle.examples import (example1_march, example1_problem, example2_march,
                             example2_problem)

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ----------------------------------------------------------------------------
# Weights (Sec. 1.2, 1.3)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("alpha", [1.1, 1.2, 1.5, 1.8, 1.9])
def test_grunwald_weights_match_library_binomial(alpha):
    g = grunwald_weights(alpha, 40)
    k = np.arange(41)
    ref = (-1.0) ** k * scipy.special.binom(alpha, k)
    np.testing.assert_allclose(g, ref, rtol=1e-13, atol=1e-16)
    assert g[0] == 1.0 and g[1] == -alpha
    assert np.all(g[2:] > 0)


@pytest.mark.parametrize("alpha", [1.2, 1.5, 1.8])
def test_grunwald_partial_sums_closed_form(alpha):
    """sum_{k<=K} (-1)^k binom(a,k) = (-1)^K binom(a-1,K); the full sum is 0."""
    K = 5000
    g = grunwald_weights(alpha, K)
    cs = np.cumsum(g)
    for Kc in (1, 2, 7, 100, 1000, 5000):
        ref = (-1.0) ** Kc * scipy.special.binom(alpha - 1.0, Kc)
        assert abs(cs[Kc] - ref) <= 1e-13 * max(1.0, abs(ref)) + 1e-16
    assert abs(cs[-1]) < 2.0 * K ** (-alpha + 0.0) * 5


@pytest.mark.parametrize("alpha", [1.2, 1.5, 1.8])
def test_wsgd_weights_sum_and_first_terms(alpha):
    w = wsgd_weights(alpha, 20000)
    g = grunwald_weights(alpha, 2)
    assert w[0] == pytest.approx(alpha / 2)
    assert w[1] == pytest.approx(alpha / 2 * g[1] + (2 - alpha) / 2 * g[0])
    assert abs(np.sum(w)) < 1e-3


# ----------------------------------------------------------------------------
# Toeplitz matrices versus the Fourier coefficients of their symbols (Sec. 2.1)
# ----------------------------------------------------------------------------

def _fourier_toeplitz(symbol, n, M=2 ** 20):
    th = 2.0 * np.pi * np.arange(M) / M
    fk = np.fft.fft(symbol(th)) / M        # (1/2pi) int f(th) e^{-ik th}
    idx = (np.arange(n)[:, None] - np.arange(n)[None, :]) % M
    return fk[idx]


@pytest.mark.parametrize("alpha", [1.2, 1.5, 1.8])
def test_T_is_toeplitz_of_symbol_g(alpha):
    """T_{alpha,n} = T_n(g_alpha): entries are the Fourier coefficients of
    g_alpha(theta) = -e^{-i theta}(1-e^{i theta})^alpha (Sec. 2.1)."""
    n = 12
    T = toeplitz_from_weights(grunwald_weights(alpha, n + 1), n)
    Tf = _fourier_toeplitz(lambda th: symbol_g(alpha, th), n)
    np.testing.assert_allclose(T, Tf.real, atol=1e-12)
    assert np.max(np.abs(Tf.imag)) < 1e-12


@pytest.mark.parametrize("alpha", [1.2, 1.5, 1.8])
def test_S_is_toeplitz_of_symbol_w(alpha):
    n = 12
    S = toeplitz_from_weights(wsgd_weights(alpha, n + 1), n)
    Sf = _fourier_toeplitz(lambda th: symbol_w(alpha, th), n)
    np.testing.assert_allclose(S, Sf.real, atol=1e-12)


def test_T_structure():
    a = 1.5
    T = toeplitz_from_weights(grunwald_weights(a, 9), 8)
    assert np.all(np.diag(T) == a)                       # -g_1
    assert np.all(np.diag(T, 1) == -1.0)                 # -g_0
    assert np.all(np.triu(T, 2) == 0.0)                  # lower Hessenberg


# ----------------------------------------------------------------------------
# Symbols (Sec. 2.2, Theorem 2, Proposition)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("alpha", [1.1, 1.3, 1.5, 1.7, 1.9])
def test_symbol_p_closed_form_and_limits(alpha):
    th = np.linspace(1e-3, np.pi, 2001)
    p = symbol_p(alpha, th)
    # derived by hand: 1 - e^{i t} = 2 sin(t/2) e^{i (t - pi)/2}
    closed = -2.0 * (2.0 * np.sin(th / 2)) ** alpha * np.cos(alpha * (th - np.pi) / 2 - th)
    np.testing.assert_allclose(p, closed, rtol=1e-12, atol=1e-14)
    assert symbol_p(alpha, np.pi) == pytest.approx(2.0 ** (alpha + 1), rel=1e-14)
    assert np.all(p > 0)
    # zero of order alpha at 0 (Proposition in Sec. 2.2)
    t = 1e-6
    assert symbol_p(alpha, t) / t ** alpha == pytest.approx(-2 * math.cos(alpha * math.pi / 2), rel=1e-5)
    # g(theta) + g(-theta) is real
    v = symbol_g(alpha, th) + symbol_g(alpha, -th)
    assert np.max(np.abs(v.imag)) < 1e-13


@pytest.mark.parametrize("alpha", [1.2, 1.5, 1.8])
def test_symbol_q_nonnegative_with_same_zero(alpha):
    th = np.linspace(1e-4, np.pi, 2001)
    q = symbol_q(alpha, th)
    assert np.all(q > 0)
    t = 1e-7
    assert symbol_q(alpha, t) / t ** alpha == pytest.approx(-2 * math.cos(alpha * math.pi / 2), rel=1e-4)
    # q_alpha(pi): w_alpha(pi) = -(1 - alpha) 2^alpha e^{0}: q = 2 (alpha - 1) 2^alpha
    assert symbol_q(alpha, np.pi) == pytest.approx(2.0 * (alpha - 1.0) * 2.0 ** alpha, rel=1e-13)


@pytest.mark.parametrize("alpha", [1.3, 1.6])
def test_symbol_p_is_fourier_series_of_T_plus_Tt(alpha):
    """p_alpha(theta) = sum_k a_k e^{ik theta}, a_k the entries of T + T^T
    (truncated at K; tail bounded by 2 sum_{k>K} g_k = -2 (-1)^K binom(a-1,K))."""
    K = 20000
    g = grunwald_weights(alpha, K + 2)
    a = np.zeros(K + 1)
    a[0] = -2 * g[1]
    a[1] = -(g[0] + g[2])
    a[2:] = -g[3:K + 2]
    th = tau_grid(31)
    series = a[0] + 2 * sum(a[k] * np.cos(k * th) for k in range(1, K + 1))
    tail = 2.0 * abs(scipy.special.binom(alpha - 1.0, K + 1))
    assert np.max(np.abs(series - symbol_p(alpha, th))) <= tail + 1e-12


# ----------------------------------------------------------------------------
# Sine transform and the tau algebra (Sec. 1)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 7, 31, 64])
def test_sine_matrix_symmetric_orthogonal_and_library_dst(n):
    S = sine_matrix(n)
    np.testing.assert_allclose(S, S.T, atol=0)
    np.testing.assert_allclose(S @ S, np.eye(n), atol=1e-13)
    import scipy.fft
    x = np.random.default_rng(n).standard_normal(n)
    np.testing.assert_allclose(S @ x, scipy.fft.dst(x, type=1, norm="ortho"), atol=1e-13)
    np.testing.assert_allclose(oracle.apply_sine_fast(x), S @ x, atol=1e-13)


def test_tau_eigenvectors():
    n = 21
    f = np.random.default_rng(1).uniform(1, 2, n)
    tau = oracle.tau_matrix(f)
    S = sine_matrix(n)
    np.testing.assert_allclose(tau @ S, S @ np.diag(f), atol=1e-13)


@pytest.mark.parametrize("n1,n2,a,b", [(7, 15, 2, 5), (15, 7, 14, 1), (2047, 3, 1000, 2), (5, 1500, 3, 777)])
@pytest.mark.parametrize("kind", ["tau_d", "d_tau_const", "shift"])
def test_tau2d_inverse_on_separable_sine_vectors(n1, n2, a, b, kind):
    """Sec. 3.2: (S (x) S) diagonalises tau(F) in 2D, so the vector
    sin(j theta_2b) sin(i theta_1a), laid out x fastest, is an eigenvector of
    P^-1 with eigenvalue 1 / (D F(theta_1a, theta_2b)).  The vector is built
    here from sin() directly; n1 != n2 catches a transposed grid, and the
    sizes above 1024 take the oracle's library-DST path."""
    alpha, beta, c0, sr = 1.5, 1.7, 0.3, 4.6
    x1 = np.arange(1, n1 + 1)[None, :] / (n1 + 1)
    x2 = np.arange(1, n2 + 1)[:, None] / (n2 + 1)
    if kind == "tau_d":
        dp, dm, ep, em = 1 + x1 + x2, 2 - x1 + 0 * x2, 1 + x1 * x2, 1 + x2 ** 2 + 0 * x1
    else:
        dp = dm = np.full((n2, n1), 1.3)
        ep = em = np.full((n2, n1), 0.9)       # D = 1.1 for the D tau order
    prob = Problem2D(alpha=alpha, beta=beta, n1=n1, n2=n2, c0=c0, sr=sr, dp=dp, dm=dm, ep=ep, em=em)
    order = ORDER_D_TAU if kind == "d_tau_const" else ORDER_TAU_D
    P = Tau2D.for_problem(prob, shift=kind == "shift", order=order)
    t1, t2 = a * np.pi / (n1 + 1), b * np.pi / (n2 + 1)
    v = (np.sin(np.arange(1, n2 + 1) * t2)[:, None] * np.sin(np.arange(1, n1 + 1) * t1)[None, :]).reshape(-1)
    qa, qb = float(symbol_q(alpha, t1)), float(symbol_q(beta, t2))
    if kind == "shift":
        lam = 1.0 / (c0 + 1.3 * qa + sr * 0.9 * qb)
    else:
        D = 0.25 * (dp + dm + ep + em)
        lam = 1.0 / ((qa + sr * qb) * D.reshape(-1))
    z = P.apply_inverse(v)
    ref = lam * v
    assert np.max(np.abs(z - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("alpha,n", [(1.5, 15), (1.2, 16), (1.8, 31)])
def test_tau_is_toeplitz_minus_hankel(alpha, n):
    """For symmetric Toeplitz A with first column c, tau(A) = A - H with the
    Hankel H_ij = c_{i+j+2} + c_{2n-i-j} (0-based, indices > n-1 dropped) is
    diagonalised by S with eigenvalues c_0 + 2 sum_{k<n} c_k cos(k theta_j);
    tau_n(p_alpha) differs from it by the aliased tail of the symbol."""
    T = toeplitz_from_weights(grunwald_weights(alpha, n + 1), n)
    A = T + T.T
    c = A[:, 0]
    H = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            for k in (i + j + 2, 2 * n - i - j):
                if 0 <= k <= n - 1:
                    H[i, j] += c[k]
    S = sine_matrix(n)
    B = S @ (A - H) @ S
    th = tau_grid(n)
    eig = c[0] + 2 * sum(c[k] * np.cos(k * th) for k in range(1, n))
    np.testing.assert_allclose(B, np.diag(eig), atol=1e-13)
    # the paper's tau_n(p_alpha) samples the full symbol: aliasing bound
    tail = 2.0 * abs(scipy.special.binom(alpha - 1.0, n))   # 2 sum_{k>=n+1} g_k
    assert np.max(np.abs(symbol_p(alpha, th) - eig)) <= tail * (1 + 1e-9)


# ----------------------------------------------------------------------------
# Solvers against LAPACK
# ----------------------------------------------------------------------------

def _const_1d_like(n, alpha=1.5):
    h = 1.0 / (n + 1)
    nu = h ** alpha / h
    return Problem1D(alpha=alpha, n=n, c0=nu, dp=np.ones(n), dm=np.ones(n), scheme=GL1)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 63])
def test_pcg_matches_lapack(n):
    prob = _const_1d_like(n)
    b = np.random.default_rng(n).uniform(-1, 1, n)
    P = Tau1D.for_problem(prob, shift=True)
    res = pcg(prob.matvec, b, Pinv=P.apply_inverse, tol=1e-14, maxiter=200)
    x = np.linalg.solve(prob.dense(), b)
    np.testing.assert_allclose(res.x, x, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("side", ["right", "left"])
@pytest.mark.parametrize("n,restart", [(3, 30), (63, 30), (127, 5)])
def test_gmres_matches_lapack(side, n, restart):
    h = 1.0 / (n + 1)
    x = h * np.arange(1, n + 1)
    prob = Problem1D(alpha=1.3, n=n, c0=h ** 1.3 * 512, dp=1 + x ** 2, dm=1 + (1 - x) ** 2)
    b = np.random.default_rng(7).uniform(-1, 1, n)
    P = Tau1D.for_problem(prob)
    res = gmres(prob.matvec, b, Pinv=P.apply_inverse, side=side, restart=restart,
                tol=1e-13, maxiter=2000)
    xs = np.linalg.solve(prob.dense(), b)
    np.testing.assert_allclose(res.x, xs, rtol=1e-9, atol=1e-12)
    assert res.converged


def test_2d_matvec_kron_and_gemm_forms_agree():
    rng = np.random.default_rng(3)
    n1, n2 = 7, 5
    prob = Problem2D(alpha=1.3, beta=1.8, n1=n1, n2=n2, c0=0.7, sr=2.5,
                     dp=rng.uniform(1, 2, (n2, n1)), dm=rng.uniform(1, 2, (n2, n1)),
                     ep=rng.uniform(1, 2, (n2, n1)), em=rng.uniform(1, 2, (n2, n1)))
    x = rng.standard_normal(n1 * n2)
    np.testing.assert_allclose(prob.matvec(x), prob.dense() @ x, atol=1e-13)
    P = Tau2D.for_problem(prob)
    np.testing.assert_allclose(P.apply_inverse(x), np.linalg.solve(P.dense(), x), atol=1e-12)


def _var_problem_2d(n1, n2, seed=4):
    rng = np.random.default_rng(seed)
    return Problem2D(alpha=1.3, beta=1.8, n1=n1, n2=n2, c0=0.7, sr=2.5,
                     dp=rng.uniform(1, 2, (n2, n1)), dm=rng.uniform(1, 2, (n2, n1)),
                     ep=rng.uniform(1, 2, (n2, n1)), em=rng.uniform(1, 2, (n2, n1)))


@pytest.mark.parametrize("n1,n2", [(7, 5), (15, 31)])
def test_2d_matvec_entries_match_kronecker_matrix(n1, n2):
    # every entry (y_j, x_i) of M x from the per-entry row sums against the
    # explicit Kronecker-product matrix (Sec. 1.4), n1 != n2 so that a swapped
    # axis or a transposed factor cannot cancel
    prob = _var_problem_2d(n1, n2)
    x = np.random.default_rng(9).standard_normal(n1 * n2)
    rows, cols = np.divmod(np.arange(n1 * n2), n1)
    got = prob.matvec_entries(x, rows, cols)
    np.testing.assert_allclose(got, prob.dense() @ x, rtol=0, atol=1e-12 * np.max(np.abs(prob.dense() @ x)))


@pytest.mark.parametrize("scheme", [GL1, WSGD2])
@pytest.mark.parametrize("n", [1, 2, 7, 300, 1023])
def test_1d_fft_convolution_path_matches_dense(n, scheme):
    rng = np.random.default_rng(n)
    prob = Problem1D(alpha=1.6, n=n, c0=0.1, dp=rng.uniform(1, 2, n), dm=rng.uniform(1, 2, n), scheme=scheme)
    x = rng.standard_normal(n)
    ref = prob.dense() @ x
    np.testing.assert_allclose(prob.matvec(x, "fft"), ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)))


def test_1d_fft_convolution_path_matches_direct_at_8191():
    rng = np.random.default_rng(8)
    n = 8191
    prob = Problem1D(alpha=1.3, n=n, c0=0.01, dp=rng.uniform(1, 2, n), dm=rng.uniform(1, 2, n))
    x = rng.standard_normal(n)
    ref = prob.matvec(x, "direct")
    np.testing.assert_allclose(prob.matvec(x, "fft"), ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))


@pytest.mark.parametrize("n1,n2", [(1, 1), (7, 5), (15, 31), (63, 127)])
def test_2d_fft_convolution_path_matches_kronecker_and_gemm_forms(n1, n2):
    prob = _var_problem_2d(n1, n2, seed=n1 + n2)
    x = np.random.default_rng(n1 * n2).standard_normal(n1 * n2)
    ref = prob.dense() @ x if n1 * n2 <= 1024 else prob.matvec(x)
    np.testing.assert_allclose(prob.matvec(x, "fft"), ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [1, 7, 255])
def test_tau1d_library_dst_path_matches_dense_sine(n):
    rng = np.random.default_rng(n + 3)
    prob = Problem1D(alpha=1.4, n=n, c0=0.2, dp=rng.uniform(1, 2, n), dm=rng.uniform(1, 2, n))
    P = Tau1D.for_problem(prob)
    r = rng.standard_normal(n)
    ref = P.apply_inverse(r)
    P.fast = True
    np.testing.assert_allclose(P.apply_inverse(r), ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))


def test_1d_direct_convolution_path_matches_dense():
    rng = np.random.default_rng(5)
    n = 300
    prob = Problem1D(alpha=1.7, n=n, c0=0.1, dp=rng.uniform(1, 2, n), dm=rng.uniform(1, 2, n))
    x = rng.standard_normal(n)
    np.testing.assert_allclose(prob.matvec(x, "direct"), prob.dense() @ x, atol=1e-12)
    rows = np.array([0, 1, 2, 150, n - 2, n - 1])
    np.testing.assert_allclose(prob.matvec_rows(x, rows), (prob.dense() @ x)[rows], atol=1e-12)


# ----------------------------------------------------------------------------
# The paper's printed numbers (Tables 1-4)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("alpha", ["1.2", "1.5", "1.8"])
@pytest.mark.parametrize("col", [0, 1, 2])
def test_table1_condition_numbers(golden, alpha, col):
    t = golden["table1_example1"]
    n = t["n_plus_1"][col] - 1
    prob, _ = example1_problem(float(alpha), n)
    M = prob.dense()
    P = Tau1D.for_problem(prob, order=ORDER_TAU_D).dense()
    assert round(preconditioned_condition_number(M, P), 1) == t["PF_kappa"][alpha][col]
    assert round(float(np.linalg.cond(M)), 1) == t["identity_kappa"][alpha][col]


@pytest.mark.parametrize("alpha", ["1.2", "1.5", "1.8"])
def test_table2_alternative_symbol_condition_numbers(golden, alpha):
    t = golden["table2_example1"]
    for col in (0, 1):
        n = t["n_plus_1"][col] - 1
        prob, _ = example1_problem(float(alpha), n)
        S = sine_matrix(n)
        F = symbol_p(float(alpha), tau_grid(n))
        D = 0.5 * (prob.dp + prob.dm)
        Pt = S @ np.diag(D * F) @ S
        assert round(preconditioned_condition_number(prob.dense(), Pt), 1) == t["PFtilde_kappa"][alpha][col]


def test_tau1d_ftilde_reproduces_table2(golden):
    """Tau1D's P_F-tilde order reproduces Table 2's printed condition numbers."""
    t = golden["table2_example1"]
    for alpha in t["PFtilde_kappa"]:
        for col in (0, 1):
            n = t["n_plus_1"][col] - 1
            prob, _ = example1_problem(float(alpha), n)
            P = Tau1D.for_problem(prob, order="tau_df").dense()
            assert round(preconditioned_condition_number(prob.dense(), P), 1) == t["PFtilde_kappa"][alpha][col]


@pytest.mark.parametrize("n", [1, 2, 9, 100])
def test_tri1d_is_the_tridiagonal_part_of_M_and_thomas_solves_it(n):
    # the diagonals against the dense M, the Thomas solve against LAPACK's
    # banded solver and the dense solve
    import scipy.linalg
    rng = np.random.default_rng(n)
    prob = Problem1D(alpha=1.6, n=n, c0=0.3, dp=rng.uniform(1, 2, n), dm=rng.uniform(1, 2, n))
    M = prob.dense()
    P = oracle.Tri1D.for_problem(prob)
    np.testing.assert_allclose(P.dense(), np.triu(np.tril(M, 1), -1), rtol=1e-14, atol=1e-14)
    r = rng.standard_normal(n)
    x = P.apply_inverse(r)
    ab = np.zeros((3, n))
    ab[0, 1:] = P.upper[:-1]
    ab[1] = P.diag
    ab[2, :-1] = P.lower[1:]
    np.testing.assert_allclose(x, scipy.linalg.solve_banded((1, 1), ab, r), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(P.dense() @ x, r, rtol=0, atol=1e-12 * np.max(np.abs(r)))


@pytest.mark.parametrize("alpha", ["1.2", "1.5", "1.8"])
def test_table2_tridiagonal_condition_numbers(golden, alpha):
    t = golden["table2_example1"]
    for col in (0, 1, 2):
        n = t["n_plus_1"][col] - 1
        prob, _ = example1_problem(float(alpha), n)
        P = oracle.Tri1D.for_problem(prob).dense()
        assert round(preconditioned_condition_number(prob.dense(), P), 1) == t["Ptri_kappa"][alpha][col]


@pytest.mark.slow
@pytest.mark.parametrize("alpha", ["1.2", "1.5", "1.8"])
def test_table2_tridiagonal_iteration_counts(golden, alpha):
    t = golden["table2_example1"]
    for col in (0, 1):
        n = t["n_plus_1"][col] - 1
        _, its, _ = example1_march(float(alpha), n, precond="tri")
        assert round(float(np.mean(its)), 1) == pytest.approx(t["Ptri_it"][alpha][col], abs=0.55)


def test_planted_missing_coefficient_breaks_tridiagonal_pin(golden):
    # d_- dropped from the off-diagonals: the printed condition number is missed
    prob, _ = example1_problem(1.5, 63)
    P = oracle.Tri1D.for_problem(prob)
    w = prob.weights()
    P.upper = -prob.dp * w[0]
    P.lower = -prob.dp * w[2]
    P.upper[-1] = 0.0
    P.lower[0] = 0.0
    k = preconditioned_condition_number(prob.dense(), P.dense())
    assert round(k, 1) != golden["table2_example1"]["Ptri_kappa"]["1.5"][0]


def test_printed_D_tau_order_does_not_reproduce_table1(golden):
    """The formula order P = D tau(F) gives 30.9 where Table 1 prints 30.8."""
    prob, _ = example1_problem(1.2, 63)
    P = Tau1D.for_problem(prob, order=ORDER_D_TAU).dense()
    k = preconditioned_condition_number(prob.dense(), P)
    assert round(k, 1) != golden["table1_example1"]["PF_kappa"]["1.2"][0]


@pytest.mark.parametrize("alpha", ["1.2", "1.5", "1.8"])
@pytest.mark.parametrize("col", [0, 1, 2])
def test_table1_iteration_counts(golden, alpha, col):
    """Left-preconditioned GMRES(20), x0 = 0, tol 1e-7 on the preconditioned
    residual, averaged over the (n+1)/2 time steps of Example 1."""
    t = golden["table1_example1"]
    n = t["n_plus_1"][col] - 1
    _, its, _ = example1_march(float(alpha), n)
    assert abs(np.mean(its) - t["PF_it"][alpha][col]) <= 0.25


@pytest.mark.parametrize("table,beta", [("table3_example2", 1.6), ("table4_example3", 1.2)])
@pytest.mark.parametrize("col", [0, 1])
def test_tables3_4_condition_numbers_and_iterations(golden, table, beta, col):
    t = golden[table]
    n = t["n"][col]
    prob, _ = example2_problem(1.8, beta, n)
    M = prob.dense()
    P = Tau2D.for_problem(prob, order=ORDER_TAU_D).dense()
    assert round(preconditioned_condition_number(M, P), 1) == t["PF_kappa"][col]
    assert round(float(np.linalg.cond(M)), 1) == t["identity_kappa"][col]
    _, its, _ = example2_march(1.8, beta, n)
    assert abs(np.mean(its) - t["PF_it"][col]) <= 0.25


# ----------------------------------------------------------------------------
# Manufactured solutions (Sec. 4.1, 4.2) and bounded iteration counts (Sec. 3)
# ----------------------------------------------------------------------------

def test_example1_first_order_convergence():
    errs = []
    for n in (63, 127, 255):
        u, _, ex = example1_march(1.5, n, tol=1e-12)
        errs.append(np.max(np.abs(u - ex)))
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(1.8 < r < 2.2 for r in ratios), (errs, ratios)


def test_example2_second_order_convergence():
    errs = []
    for n in (15, 31):
        u, _, ex = example2_march(1.8, 1.6, n, tol=1e-12)
        errs.append(np.max(np.abs(u - ex)))
    assert errs[0] / errs[1] > 3.3, errs


def test_case1_shifted_pcg_iterations_bounded_in_n():
    """Case I (Sec. 3.1.1): the shifted tau preconditioner keeps PCG iteration
    counts flat as n grows (config-1 shape: alpha=1.5, d=1, dt=h)."""
    its = []
    for n in (63, 255, 1023, 4095):
        prob = _const_1d_like(n)
        b = np.random.default_rng(0).uniform(-1, 1, n)
        P = Tau1D.for_problem(prob, shift=True)
        res = pcg(prob.matvec, b, Pinv=P.apply_inverse, tol=1e-8)
        assert res.converged and res.relres <= 1e-8
        its.append(res.iterations)
    assert max(its) <= 6 and max(its) - min(its) <= 1, its


def test_shifted_variable_coefficient_variant_bounded_and_cheaper():
    """The shift nu/dbar kept beside a variable D (the variable-coefficient
    generalisation of Case I) on the variable-coefficient workload shape at
    alpha = 1.2, where nu dominates the lowest symbol samples: GMRES
    iterations grow at most logarithmically in n (8, 11, 13 for n = 255,
    1023, 4095) and stay below half those of the unshifted P_F (29, 38, 44)."""
    import workloads
    its_s, its_u = [], []
    for n in (255, 1023, 4095):
        w = workloads.var_1d_time_stepping(n=n, alphas=(1.2,))[0]
        h = 1.0 / (n + 1)
        prob = Problem1D(alpha=1.2, n=n, c0=h ** 1.2 / w["dt"], dp=w["dp"], dm=w["dm"])
        b = prob.c0 * w["u0"]
        for shift, its in ((True, its_s), (False, its_u)):
            P = Tau1D.for_problem(prob, shift=shift)
            res = gmres(prob.matvec, b, Pinv=P.apply_inverse, restart=30, tol=1e-8, maxiter=2000)
            assert res.converged
            its.append(res.iterations)
    assert its_s == sorted(its_s) and its_s[-1] - its_s[0] <= 6 and its_s[-1] <= 16, its_s
    assert all(s * 2 <= u for s, u in zip(its_s, its_u)), (its_s, its_u)


def test_2d_shifted_pcg_iterations_bounded_in_n():
    """Theorem 3: P_hat gives a spectrum bounded independently of N."""
    its = []
    for n in (63, 255):
        h = 1.0 / (n + 1)
        a, b_ = 1.5, 1.7
        one = np.ones((n, n))
        prob = Problem2D(alpha=a, beta=b_, n1=n, n2=n, c0=h ** a / h, sr=h ** a / h ** b_,
                         dp=one, dm=one, ep=one, em=one, scheme=WSGD2)
        rhs = np.random.default_rng(1).uniform(-1, 1, n * n)
        P = Tau2D.for_problem(prob, shift=True)
        res = pcg(prob.matvec, rhs, Pinv=P.apply_inverse, tol=1e-8)
        assert res.converged
        its.append(res.iterations)
    assert max(its) <= 7 and max(its) - min(its) <= 1, its


# ----------------------------------------------------------------------------
# Planted mistakes: the pins above must catch plausible errors in the oracle
# ----------------------------------------------------------------------------

def test_planted_transposed_T_breaks_table1_pin(golden, monkeypatch):
    prob, _ = example1_problem(1.5, 63)
    T = prob.T()
    prob._T = T.T.copy()                      # plant: swap T and T^T
    k = preconditioned_condition_number(prob.dense(), Tau1D.for_problem(prob).dense())
    assert round(k, 1) != golden["table1_example1"]["PF_kappa"]["1.5"][0]


def test_planted_sign_error_in_weights_breaks_fourier_pin(monkeypatch):
    n, alpha = 12, 1.5
    g = grunwald_weights(alpha, n + 1)
    g_bad = np.abs(g)                         # plant: drop the (-1)^k
    T = toeplitz_from_weights(g_bad, n)
    Tf = _fourier_toeplitz(lambda th: symbol_g(alpha, th), n)
    assert np.max(np.abs(T - Tf.real)) > 1e-3


def test_planted_index_shift_breaks_hankel_pin():
    n = 15
    T = toeplitz_from_weights(grunwald_weights(1.5, n + 1), n)
    A = T + T.T
    c = A[:, 0]
    H = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            for k in (i + j, 2 * n - 2 - i - j):       # plant: off-by-one indices
                if 0 <= k <= n - 1:
                    H[i, j] += c[k]
    S = sine_matrix(n)
    B = S @ (A - H) @ S
    assert np.max(np.abs(B - np.diag(np.diag(B)))) > 1e-3


@pytest.mark.parametrize("plant", ["x_transposed", "y_transposed", "axes_swapped"])
def test_planted_mistakes_break_matvec_entries_pin(plant):
    # T^T for T on the x lines (Ta[i] <-> Ta[:, i]), the same on the y lines,
    # or the coefficient arrays of the two axes exchanged: each changes entries
    # of M x that the Kronecker matrix fixes
    n1, n2 = 7, 5
    prob = _var_problem_2d(n1, n2)
    x = np.random.default_rng(9).standard_normal(n1 * n2)
    U = x.reshape(n2, n1)
    Ta, Tb = prob.Ta(), prob.Tb()
    rows, cols = np.divmod(np.arange(n1 * n2), n1)
    bad = np.empty(n1 * n2)
    for t, (j, i) in enumerate(zip(rows, cols)):
        if plant == "x_transposed":
            ax = prob.dp[j, i] * (Ta[:, i] @ U[j]) + prob.dm[j, i] * (Ta[i] @ U[j])
        else:
            ax = prob.dp[j, i] * (Ta[i] @ U[j]) + prob.dm[j, i] * (Ta[:, i] @ U[j])
        if plant == "y_transposed":
            ay = prob.ep[j, i] * (Tb[:, j] @ U[:, i]) + prob.em[j, i] * (Tb[j] @ U[:, i])
        else:
            ay = prob.ep[j, i] * (Tb[j] @ U[:, i]) + prob.em[j, i] * (Tb[:, j] @ U[:, i])
        if plant == "axes_swapped":
            ax, ay = (prob.ep[j, i] * (Ta[i] @ U[j]) + prob.em[j, i] * (Ta[:, i] @ U[j]),
                      prob.dp[j, i] * (Tb[j] @ U[:, i]) + prob.dm[j, i] * (Tb[:, j] @ U[:, i]))
        bad[t] = prob.c0 * U[j, i] + ax + prob.sr * ay
    ref = prob.dense() @ x
    assert np.max(np.abs(bad - ref)) > 1e-3 * np.max(np.abs(ref))
    np.testing.assert_allclose(prob.matvec_entries(x, rows, cols), ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))


def test_planted_missing_shift_breaks_bounded_iterations():
    n = 1023
    prob = _const_1d_like(n)
    b = np.random.default_rng(0).uniform(-1, 1, n)
    P = Tau1D.for_problem(prob, shift=False)      # plant: unshifted symbol
    res = pcg(prob.matvec, b, Pinv=P.apply_inverse, tol=1e-8)
    assert res.iterations > 10
