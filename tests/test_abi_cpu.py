"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point of include/fde.h, and validates arguments before launching."""

import ctypes

import pytest

import paper_1912_13304_gb300 as fde


@pytest.fixture(scope="module")
def L():
    from paper_1912_13304_gb300 import build
    build.build()
    return fde.lib()


def test_every_header_symbol_is_exported(L):
    names = fde.header_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(L, name), name


def test_status_strings(L):
    for s in range(8):
        assert fde.status_string(s)
    assert fde.status_string(fde.EINVAL) == "invalid argument"


def test_default_opts(L):
    o = fde.default_opts()
    assert o.method == fde.GMRES and o.restart == 30 and o.tol == 1e-8 and o.precision == fde.PREC_F64


def _ws(p, o):
    n = ctypes.c_size_t(0)
    st = fde.lib().fde_workspace_size(ctypes.byref(p), ctypes.byref(o), ctypes.byref(n))
    return st, n.value


def test_workspace_size_valid_problems(L):
    o = fde.make_opts(method="pcg")
    p = fde.make_problem(1, 1023, 1.5, 1.0 / 1024, tau_shift=True)
    st, n = _ws(p, o)
    assert st == fde.OK and n > 1023 * 8
    o2 = fde.make_opts(method="gmres", restart=20, precision="f32_ir")
    p2 = fde.make_problem(2, 63, 1.3, 1 / 256., n2=127, beta=1.8, weights="wsgd2", dp=1 << 20, dm=2 << 20,
                          ep=3 << 20, em=4 << 20)
    st, n2 = _ws(p2, o2)
    assert st == fde.OK and n2 > 63 * 127 * (20 + 6) * 4


@pytest.mark.parametrize("field,value", [
    ("n1", 0), ("n1", 1000), ("alpha", 1.0), ("alpha", 2.0), ("alpha", float("nan")), ("dt", 0.0),
    ("len1", -1.0), ("dim", 3), ("weights", 5), ("order", 4), ("scheme", 7),
])
def test_invalid_problem_rejected(L, field, value):
    o = fde.make_opts()
    p = fde.make_problem(1, 255, 1.5, 0.01)
    setattr(p, field, value)
    st, _ = _ws(p, o)
    assert st == fde.EINVAL


def test_tridiagonal_preconditioner_is_1d_and_unshifted(L):
    o = fde.make_opts()
    assert _ws(fde.make_problem(1, 255, 1.5, 0.01, order="tri"), o)[0] == fde.OK
    assert _ws(fde.make_problem(1, 255, 1.5, 0.01, order="tri", tau_shift=True), o)[0] == fde.EINVAL
    p2 = fde.make_problem(2, 63, 1.3, 0.01, n2=63, beta=1.8, weights="wsgd2", order="tri")
    assert _ws(p2, o)[0] == fde.EINVAL


@pytest.mark.parametrize("field,value", [
    ("restart", 0), ("restart", 65), ("tol", 0.0), ("max_iters", 0), ("precision", 3), ("side", 2),
    ("method", 9),
])
def test_invalid_opts_rejected(L, field, value):
    o = fde.make_opts()
    setattr(o, field, value)
    st, _ = _ws(fde.make_problem(1, 255, 1.5, 0.01), o)
    assert st == fde.EINVAL


def test_ftilde_order_is_1d_and_unshifted(L):
    o = fde.make_opts()
    st, _ = _ws(fde.make_problem(1, 255, 1.5, 0.01, dp=1 << 20, dm=1 << 20, order="tau_df"), o)
    assert st == fde.OK
    st, _ = _ws(fde.make_problem(2, 63, 1.5, 0.01, n2=63, beta=1.5, order="tau_df"), o)
    assert st == fde.EINVAL
    st, _ = _ws(fde.make_problem(1, 255, 1.5, 0.01, order="tau_df", tau_shift=True), o)
    assert st == fde.EINVAL


def test_pcg_needs_symmetric_constant_problem(L):
    o = fde.make_opts(method="pcg")
    # variable coefficients: P = tau D is not symmetric
    st, _ = _ws(fde.make_problem(1, 255, 1.5, 0.01, dp=1 << 20, dm=1 << 20), o)
    assert st == fde.EINVAL
    # d_+ != d_-: M is not symmetric
    st, _ = _ws(fde.make_problem(1, 255, 1.5, 0.01, dp_const=1.0, dm_const=2.0, tau_shift=True), o)
    assert st == fde.EINVAL
    st, _ = _ws(fde.make_problem(1, 255, 1.5, 0.01, dp_const=2.0, dm_const=2.0, tau_shift=True), o)
    assert st == fde.OK


def test_shift_with_variable_coefficients_1d_gmres_only(L):
    # 1D: the shift c0/mean(D) beside a variable D is a GMRES preconditioner
    st, _ = _ws(fde.make_problem(1, 255, 1.5, 0.01, dp=1 << 20, dm=1 << 20, tau_shift=True), fde.make_opts())
    assert st == fde.OK
    # ... not symmetric, so not for PCG
    st, _ = _ws(fde.make_problem(1, 255, 1.5, 0.01, dp=1 << 20, dm=1 << 20, tau_shift=True),
                fde.make_opts(method="pcg"))
    assert st == fde.EINVAL
    # 2D: P_hat needs constant coefficients
    st, _ = _ws(fde.make_problem(2, 255, 1.5, 0.01, n2=255, beta=1.5, dp=1 << 20, dm=1 << 20, tau_shift=True),
                fde.make_opts())
    assert st == fde.EINVAL


def test_2d_size_limit(L):
    o = fde.make_opts()
    st, _ = _ws(fde.make_problem(2, 8191, 1.5, 0.01, n2=63, beta=1.5), o)
    assert st == fde.EINVAL


def test_calls_reject_null_arguments_without_launching(L):
    assert L.fde_toeplitz_matvec(None, 0, None, None, None) == fde.EINVAL
    assert L.fde_tau_solve(None, 0, None, None, None) == fde.EINVAL
    o = fde.make_opts()
    assert L.fde_krylov_solve(None, 1, None, None, ctypes.byref(o), None, None) == fde.EINVAL
    h = ctypes.c_void_p(0)
    p = fde.make_problem(1, 255, 1.5, 0.01)
    assert L.fde_assemble_symbol(ctypes.byref(p), ctypes.byref(o), None, 0, ctypes.byref(h), None) == fde.EINVAL
    assert L.fde_step_rhs(None, None, None, None, None) == fde.EINVAL


def test_assembly_rejects_a_short_workspace_before_any_launch(L):
    p = fde.make_problem(1, 1023, 1.5, 0.01)
    o = fde.make_opts()
    st, need = _ws(p, o)
    assert st == fde.OK
    plan = ctypes.c_void_p()
    # a 256-byte aligned address that is never dereferenced: the size check comes first
    st = L.fde_assemble_symbol(ctypes.byref(p), ctypes.byref(o), 1 << 20, need - 1, ctypes.byref(plan), 0)
    assert st == fde.ENOMEM and not plan.value
