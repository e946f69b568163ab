"""The paper's numerical examples (Sec. 4), built with the oracle's plain FP64
definitions.  TEST INFRASTRUCTURE ONLY.

Example 1 (Sec. 4.1): 1D on [0,2] x [0,1], d_+ = Gamma(3-a) x^a,
d_- = Gamma(3-a)(2-x)^a, h_x = h_t = 2/(n+1), nu = h^(a-1), M = (n+1)/2
implicit-Euler steps, exact solution u = 4 e^{-t} x^2 (2-x)^2.

Examples 2 and 3 (Sec. 4.2, 4.3): 2D on [0,2]^2, Crank-Nicolson with the WSGD
weights, n1 = n2 = n = M time steps.  The step size is read as h_t = 1/M
(the text also writes 1/(M+1); only 1/M reproduces the tabulated condition
numbers and matches M steps over [0, 1]).
"""

from __future__ import annotations

import math

import numpy as np

from .fde_oracle import (GL1, WSGD2, ORDER_TAU_D, Problem1D, Problem2D, Tau1D, Tau2D, Tri1D,
                         gmres)


# ----------------------------------------------------------------------------
# Example 1
# ----------------------------------------------------------------------------

def example1_problem(alpha: float, n: int) -> tuple[Problem1D, dict]:
    h = 2.0 / (n + 1)
    x = h * np.arange(1, n + 1)
    g3 = math.gamma(3.0 - alpha)
    dp = g3 * x ** alpha
    dm = g3 * (2.0 - x) ** alpha
    nu = h ** alpha / h            # h_t = h
    prob = Problem1D(alpha=alpha, n=n, c0=nu, dp=dp, dm=dm, scheme=GL1)
    meta = dict(h=h, ht=h, steps=(n + 1) // 2, x=x)
    return prob, meta


def example1_source(alpha: float, x: np.ndarray, t: float) -> np.ndarray:
    a = alpha
    return -32.0 * math.exp(-t) * (
        x ** 2 + (2 - x) ** 2 * (8 + x ** 2) / 8.0
        - 3.0 * (x ** 3 + (2 - x) ** 3) / (3.0 - a)
        + 3.0 * (x ** 4 + (2 - x) ** 4) / ((4.0 - a) * (3.0 - a)))


def example1_exact(x: np.ndarray, t: float) -> np.ndarray:
    return 4.0 * math.exp(-t) * x ** 2 * (2 - x) ** 2


def example1_march(alpha: float, n: int, precond: str = "PF", order: str = ORDER_TAU_D,
                   side: str = "left", restart: int = 20, tol: float = 1e-7,
                   warm_start: bool = False):
    """Implicit Euler over [0, 1] with GMRES per step (Sec. 1.2, Sec. 4.1).

    Returns (u_final, list of iteration counts, exact u at T=1).
    """
    prob, meta = example1_problem(alpha, n)
    x, h, ht, M = meta["x"], meta["h"], meta["ht"], meta["steps"]
    P = None
    if precond == "PF":
        P = Tau1D.for_problem(prob, shift=False, order=order).apply_inverse
    elif precond == "tri":
        P = Tri1D.for_problem(prob).apply_inverse
    u = example1_exact(x, 0.0)
    its = []
    for m in range(1, M + 1):
        t = m * ht
        b = prob.c0 * u + h ** alpha * example1_source(alpha, x, t)
        res = gmres(prob.matvec, b, Pinv=P, x0=(u if warm_start else None), side=side,
                    restart=restart, tol=tol)
        u = res.x
        its.append(res.iterations)
    return u, its, example1_exact(x, M * ht)


# ----------------------------------------------------------------------------
# Examples 2 and 3
# ----------------------------------------------------------------------------

def example2_problem(alpha: float, beta: float, n: int) -> tuple[Problem2D, dict]:
    h = 2.0 / (n + 1)
    M = n
    ht = 1.0 / M
    xs = h * np.arange(1, n + 1)
    X, Y = np.meshgrid(xs, xs, indexing="xy")      # X[j, i] = x_i, Y[j, i] = y_j
    ga, gb = math.gamma(3.0 - alpha), math.gamma(3.0 - beta)
    dp = ga * (1 + X) ** alpha * (1 + Y) ** 2
    dm = ga * (3 - X) ** alpha * (3 - Y) ** 2
    ep = gb * (1 + X) ** 2 * (1 + Y) ** beta
    em = gb * (3 - X) ** 2 * (3 - Y) ** beta
    r = ht / (2.0 * h ** alpha)
    s = ht / (2.0 * h ** beta)
    prob = Problem2D(alpha=alpha, beta=beta, n1=n, n2=n, c0=1.0 / r, sr=s / r,
                     dp=dp, dm=dm, ep=ep, em=em, scheme=WSGD2)
    return prob, dict(h=h, ht=ht, steps=M, X=X, Y=Y)


def _g_gamma(gam: float, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    return ((8 * x ** (2 - gam) - 24 * x ** (3 - gam) / (3 - gam)
             + 24 * x ** (4 - gam) / ((4 - gam) * (3 - gam)))
            * (1 + x) ** gam * (1 + y) ** 2 * y ** 2 * (2 - y) ** 2)


def example2_source(alpha, beta, X, Y, t):
    return -16.0 * math.exp(-t) * (
        X ** 2 * (2 - X) ** 2 * Y ** 2 * (2 - Y) ** 2
        + _g_gamma(alpha, X, Y) + _g_gamma(alpha, 2 - X, 2 - Y)
        + _g_gamma(beta, Y, X) + _g_gamma(beta, 2 - Y, 2 - X))


def example2_exact(X, Y, t):
    return 16.0 * math.exp(-t) * X ** 2 * (2 - X) ** 2 * Y ** 2 * (2 - Y) ** 2


def example2_march(alpha: float, beta: float, n: int, precond: str = "PF",
                   order: str = ORDER_TAU_D, side: str = "left", restart: int = 20,
                   tol: float = 1e-7):
    """Crank-Nicolson steps (Sec. 1.4):
    M u^m = (1/r I - A_x - (s/r) A_y) u^{m-1} + 2 h^alpha f(t_{m-1/2}),
    where the explicit operator equals 2 (1/r) u - M u."""
    prob, meta = example2_problem(alpha, beta, n)
    X, Y, h, ht, M = meta["X"], meta["Y"], meta["h"], meta["ht"], meta["steps"]
    P = None
    if precond == "PF":
        P = Tau2D.for_problem(prob, shift=False, order=order).apply_inverse
    u = example2_exact(X, Y, 0.0).reshape(-1)
    its = []
    for m in range(1, M + 1):
        tm = (m - 0.5) * ht
        b = (2.0 * prob.c0 * u - prob.matvec(u)
             + 2.0 * h ** alpha * example2_source(alpha, beta, X, Y, tm).reshape(-1))
        res = gmres(prob.matvec, b, Pinv=P, side=side, restart=restart, tol=tol)
        u = res.x
        its.append(res.iterations)
    return u, its, example2_exact(X, Y, M * ht).reshape(-1)
