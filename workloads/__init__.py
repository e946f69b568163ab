"""Seeded synthetic inputs shaped like the five benchmark workloads (1D constant
coefficients, 1D variable-coefficient time stepping, 2D constant coefficients,
a batch of 1D constant-coefficient solves, 2D variable-coefficient time stepping).

This module is shared by the oracle and the CUDA path and holds none of the
method's arithmetic: it only lays out grids, evaluates the coefficient and
initial-data functions of each workload on the grid, and draws seeded random
numbers (numpy PCG64 via ``default_rng``, draw order documented per workload).

Conventions: grids are interior points x_i = i h, i = 1..n, h = length/(n+1);
2D arrays have shape (n2, n1) with x fastest (element [j, i] = value at
(x_i, y_j)), matching the paper's ordering u[i + j n1].  ``rhs_scale`` names
how the workload states its right-hand side: "unit" means the system was
written as (I + dt h^-alpha (...)) u = b, i.e. the paper's M u = c0 b.
"""

from __future__ import annotations

import numpy as np


def grid(n: int, length: float = 1.0):
    h = length / (n + 1)
    return h, h * np.arange(1, n + 1, dtype=np.float64)


def const_1d(n: int = 1023, alpha: float = 1.5, seed: int = 0) -> dict:
    """1D constant coefficients d+ = d- = 1 on [0,1], one implicit-Euler step
    with dt = h, rhs uniform[-1,1] (seed 0, n draws), PCG with the shifted
    (Case I) tau preconditioner, relres 1e-8, FP64."""
    h, x = grid(n)
    rng = np.random.default_rng(seed)
    b = rng.uniform(-1.0, 1.0, n)
    return dict(name=f"1d-const-n{n}", dim=1, n1=n, n2=1, alpha=alpha, beta=alpha,
                length=1.0, dt=h, dp=np.ones(n), dm=np.ones(n), const_coeffs=True,
                b=b, rhs_scale="unit", scheme="gl1", method="pcg", shift=True,
                order="tau_d", restart=0, tol=1e-8, steps=1)


def var_1d_time_stepping(n: int = 65535, alphas=(1.2, 1.5, 1.8), steps: int = 20, dt: float = 1.0 / 512,
            seed: int = 0) -> list[dict]:
    """1D variable coefficients d+ = 1 + x^2, d- = 1 + (1-x)^2 on [0,1],
    implicit Euler with dt = 1/512, u0 = x^2 (1-x)^2 + uniform[-1e-3, 1e-3]
    noise (seed 0, n draws, shared by every alpha), f = 0, GMRES(30) with the
    unshifted tau preconditioner (tau D order)."""
    h, x = grid(n)
    rng = np.random.default_rng(seed)
    u0 = x ** 2 * (1 - x) ** 2 + rng.uniform(-1e-3, 1e-3, n)
    out = []
    for a in alphas:
        out.append(dict(name=f"1d-var-n{n}-a{a}", dim=1, n1=n, n2=1, alpha=a, beta=a,
                        length=1.0, dt=dt, dp=1 + x ** 2, dm=1 + (1 - x) ** 2,
                        const_coeffs=False, u0=u0.copy(), rhs_scale="step",
                        scheme="gl1", method="gmres", shift=False, order="tau_d",
                        restart=30, tol=1e-8, steps=steps))
    return out


def const_2d(n: int = 2047, alpha: float = 1.5, beta: float = 1.7, seed: int = 1) -> dict:
    """2D constant coefficients d+- = e+- = 1 on the unit square, one implicit
    step with dt = h, rhs uniform[-1,1] (seed 1, N draws, x fastest), WSGD
    weights, PCG with P_hat (shifted, no D)."""
    h, x = grid(n)
    rng = np.random.default_rng(seed)
    b = rng.uniform(-1.0, 1.0, n * n)
    one = np.ones((n, n))
    return dict(name=f"2d-const-n{n}", dim=2, n1=n, n2=n, alpha=alpha, beta=beta,
                length=1.0, dt=h, dp=one, dm=one, ep=one, em=one, const_coeffs=True,
                b=b, rhs_scale="unit", scheme="wsgd2", method="pcg", shift=True,
                order="tau_d", restart=0, tol=1e-8, steps=1)


def const_1d_batch(count: int = 256, kmin: int = 8, kmax: int = 14, seed: int = 2) -> list[dict]:
    """Independent 1D constant-coefficient solves.  For each instance, in order,
    from one generator (seed 2): k ~ U{kmin..kmax} (n = 2^k - 1),
    alpha ~ U(1.1, 1.9), d ~ U[0.5, 2] (d+ = d- = d), dt = U[0.5, 2] * h, then
    n rhs values ~ U[-1, 1]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        k = int(rng.integers(kmin, kmax + 1))
        alpha = float(rng.uniform(1.1, 1.9))
        d = float(rng.uniform(0.5, 2.0))
        dtf = float(rng.uniform(0.5, 2.0))
        n = 2 ** k - 1
        h, _ = grid(n)
        b = rng.uniform(-1.0, 1.0, n)
        out.append(dict(name=f"batch{i}-n{n}", dim=1, n1=n, n2=1, alpha=alpha, beta=alpha,
                        length=1.0, dt=dtf * h, dp=np.full(n, d), dm=np.full(n, d),
                        const_coeffs=True, b=b, rhs_scale="unit", scheme="gl1",
                        method="pcg", shift=True, order="tau_d", restart=0, tol=1e-8,
                        steps=1))
    return out


def var_2d_time_stepping(n: int = 4095, alpha: float = 1.3, beta: float = 1.8, steps: int = 50,
            dt: float = 1.0 / 256) -> dict:
    """2D variable coefficients d+ = 1+x+y, d- = 2-x, e+ = 1+xy, e- = 1+y^2 on
    the unit square, u0 = sin(pi x) sin(pi y), f = 0, implicit Euler dt = 1/256,
    WSGD weights, GMRES(20) with the unshifted 2D tau preconditioner and D_N."""
    h, x = grid(n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    return dict(name=f"2d-var-n{n}", dim=2, n1=n, n2=n, alpha=alpha, beta=beta,
                length=1.0, dt=dt, dp=1 + X + Y, dm=2 - X, ep=1 + X * Y, em=1 + Y ** 2,
                const_coeffs=False, u0=(np.sin(np.pi * X) * np.sin(np.pi * Y)).reshape(-1),
                rhs_scale="step", scheme="wsgd2", method="gmres", shift=False,
                order="tau_d", restart=20, tol=1e-8, steps=steps)
