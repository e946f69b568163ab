"""fde_toeplitz_matvec_noalloc: y = M x for a 1D problem with its scratch in a
fixed static device array.  Its results must agree with the plan-based
fde_toeplitz_matvec on the same problem and input, call after call.

The file name sorts last so that the GPU test also runs after every other
test has used the device."""

import ctypes

import numpy as np
import pytest

import paper_1912_13304_gb300 as fde


@pytest.fixture(scope="module")
def L():
    from paper_1912_13304_gb300 import build
    build.build()
    return fde.lib()


def _call(L, prob, x, y):
    return L.fde_toeplitz_matvec_noalloc(ctypes.byref(prob), x, y, 0)


def test_rejects_sizes_beyond_the_scratch(L):
    # checked before any CUDA call: the pointers are never dereferenced
    assert fde.MATVEC_NOALLOC_MAX_N == 4095
    assert _call(L, fde.make_problem(1, 8191, 1.5, 0.01), 16, 32) == fde.ENOMEM


def test_rejects_invalid_arguments(L):
    prob = fde.make_problem(1, 255, 1.5, 0.01)
    assert _call(L, prob, 16, 16) == fde.EINVAL               # x == y
    assert _call(L, prob, 0, 32) == fde.EINVAL                # NULL x
    assert L.fde_toeplitz_matvec_noalloc(None, 16, 32, 0) == fde.EINVAL
    assert _call(L, fde.make_problem(2, 255, 1.5, 0.01, n2=255, beta=1.5), 16, 32) == fde.EINVAL
    assert _call(L, fde.make_problem(1, 254, 1.5, 0.01), 16, 32) == fde.EINVAL     # n + 1 not 2^k
    assert _call(L, fde.make_problem(1, 255, 2.5, 0.01), 16, 32) == fde.EINVAL     # alpha outside (1, 2)


@pytest.mark.gpu
def test_matches_plan_matvec_two_calls_in_a_row(gpu):
    import torch

    import oracle

    # Rounding order differs (global-memory radix-8 passes against the
    # engine's shared-memory transforms); both are FP64 FFT products whose
    # error is a few ulps times log2(L) relative to the largest entry.  The
    # oracle's dense product from the weights is the reference of both.
    tol = 1e-12
    rng = np.random.default_rng(7)
    cases = []
    for n, alpha, weights, scheme, variable in [(4095, 1.7, "gl1", "ie", True), (255, 1.3, "wsgd2", "cn", False),
                                                (1, 1.5, "gl1", "ie", True)]:
        h = 1.0 / (n + 1)
        dt = 1.0 / 256
        xg = h * np.arange(1, n + 1)
        kw = dict(weights=weights, scheme=scheme)
        if variable:
            dp, dm = 1 + xg ** 2, 1 + (1 - xg) ** 2
            kw.update(dp=dp, dm=dm)
        else:
            dp = dm = np.full(n, 0.7)
            kw.update(dp_const=0.7, dm_const=0.7)
        plan = fde.Plan(1, n, alpha, dt, **kw)
        xh = rng.uniform(-1, 1, n)
        x = torch.tensor(xh, device="cuda", dtype=torch.float64)
        c0 = (2.0 if scheme == "cn" else 1.0) * h ** alpha / dt
        prob = oracle.Problem1D(alpha=alpha, n=n, c0=c0, dp=dp, dm=dm, scheme=weights)
        cases.append((plan, x, plan.matvec(x), prob.matvec(xh, "dense")))
    torch.cuda.synchronize()
    for rep in range(2):
        for plan, x, ref, ref_oracle in cases:
            y = torch.full_like(x, float("nan"))
            fde.toeplitz_matvec_noalloc(plan.problem, x, y)
            torch.cuda.synchronize()
            err = (y - ref).abs().max().item() / ref.abs().max().item()
            assert err < tol, (rep, plan.n1, err)
            yh = y.cpu().numpy()
            err_o = np.max(np.abs(yh - ref_oracle)) / np.max(np.abs(ref_oracle))
            assert err_o < tol, (rep, plan.n1, err_o)
