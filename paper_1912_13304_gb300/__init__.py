"""Python binding of libfde (include/fde.h): argument marshalling only.

Every computation of the solve path runs in the CUDA kernels of libfde.so;
this module converts Python values to the C structs, passes device pointers
(torch CUDA tensors or raw integers) and streams, and keeps the tensors that a
plan depends on alive.  There is no CPU fallback: if the shared library is
missing, ``lib()`` raises.
"""

from __future__ import annotations

import ctypes
import os
import re
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfde.so")
HEADER = os.path.join(HERE, "..", "include", "fde.h")

# enums (include/fde.h)
OK, EINVAL, ENOMEM, ECUDA, ENOCONV, EBREAKDOWN, ETIMEOUT, ENONFINITE = range(8)
F64, F32 = 0, 1
WEIGHTS_GL1, WEIGHTS_WSGD2 = 0, 1
ORDER_TAU_D, ORDER_D_TAU, ORDER_TAU_DF, ORDER_TRI = 0, 1, 2, 3
SCHEME_IMPLICIT_EULER, SCHEME_CRANK_NICOLSON = 0, 1
PCG, GMRES = 0, 1
PREC_F64, PREC_F32, PREC_F32_IR = 0, 1, 2
SIDE_RIGHT, SIDE_LEFT = 0, 1


class FdeProblem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n1", ctypes.c_int), ("n2", ctypes.c_int),
        ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
        ("len1", ctypes.c_double), ("len2", ctypes.c_double), ("dt", ctypes.c_double),
        ("scheme", ctypes.c_int), ("weights", ctypes.c_int),
        ("dp", ctypes.c_void_p), ("dm", ctypes.c_void_p), ("ep", ctypes.c_void_p), ("em", ctypes.c_void_p),
        ("dp_const", ctypes.c_double), ("dm_const", ctypes.c_double),
        ("ep_const", ctypes.c_double), ("em_const", ctypes.c_double),
        ("tau_shift", ctypes.c_int), ("order", ctypes.c_int),
    ]


class FdeSolveOpts(ctypes.Structure):
    _fields_ = [
        ("method", ctypes.c_int), ("restart", ctypes.c_int), ("tol", ctypes.c_double),
        ("max_iters", ctypes.c_int), ("precision", ctypes.c_int), ("inner_tol", ctypes.c_double),
        ("max_outer", ctypes.c_int), ("side", ctypes.c_int), ("balance", ctypes.c_int),
    ]


class FdeSolveInfo(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32), ("iterations", ctypes.c_int32), ("outer", ctypes.c_int32),
        ("restarts", ctypes.c_int32), ("relres", ctypes.c_double), ("relres_est", ctypes.c_double),
        ("basis_sum", ctypes.c_int32), ("reorth", ctypes.c_int32), ("cycles", ctypes.c_int32),
        ("residuals64", ctypes.c_int32), ("iterations64", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


INFO_BYTES = ctypes.sizeof(FdeSolveInfo)
_lib = None


class FdeError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


def lib() -> ctypes.CDLL:
    """Load libfde.so (built by build.py / __graft_entry__.build()).  Raises if missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfde.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, cint, cdbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        P = ctypes.POINTER
        L.fde_default_opts.argtypes = [P(FdeSolveOpts)]
        L.fde_default_opts.restype = None
        L.fde_workspace_size.argtypes = [P(FdeProblem), P(FdeSolveOpts), P(ctypes.c_size_t)]
        L.fde_workspace_size.restype = cint
        L.fde_assemble_symbol.argtypes = [P(FdeProblem), P(FdeSolveOpts), vp, ctypes.c_size_t, P(vp), vp]
        L.fde_assemble_symbol.restype = cint
        L.fde_toeplitz_matvec.argtypes = [vp, cint, vp, vp, vp]
        L.fde_toeplitz_matvec.restype = cint
        L.fde_selftest_barrier_timeout.argtypes = [vp, vp, vp]
        L.fde_selftest_barrier_timeout.restype = cint
        L.fde_plan_set_schedule.argtypes = [vp, cint, cint, vp]
        L.fde_plan_set_schedule.restype = cint
        L.fde_autotune.argtypes = [vp, vp, P(cint), P(cint)]
        L.fde_autotune.restype = cint
        L.fde_toeplitz_matvec_noalloc.argtypes = [P(FdeProblem), vp, vp, vp]
        L.fde_toeplitz_matvec_noalloc.restype = cint
        L.fde_tau_solve.argtypes = [vp, cint, vp, vp, vp]
        L.fde_tau_solve.restype = cint
        L.fde_krylov_solve.argtypes = [P(vp), cint, P(vp), P(vp), P(FdeSolveOpts), vp, vp]
        L.fde_krylov_solve.restype = cint
        L.fde_step_rhs.argtypes = [vp, vp, vp, vp, vp]
        L.fde_step_rhs.restype = cint
        L.fde_measure_fp64_rate.argtypes = [P(cdbl), vp]
        L.fde_measure_fp64_rate.restype = cint
        L.fde_plan_scalars.argtypes = [vp, P(cdbl), P(cdbl), P(cdbl)]
        L.fde_plan_scalars.restype = cint
        L.fde_plan_destroy.argtypes = [vp]
        L.fde_plan_destroy.restype = None
        L.fde_status_string.argtypes = [cint]
        L.fde_status_string.restype = ctypes.c_char_p
        _lib = L
    return _lib


def header_functions() -> list[str]:
    """Names of the entry points declared in include/fde.h."""
    with open(HEADER) as f:
        text = f.read()
    pat = r"^\s*(?:fde_status|void|const\s+char\s*\*)\s*(fde_[a-z_0-9]+)\s*\("
    return sorted(set(re.findall(pat, text, flags=re.M)))


def status_string(status: int) -> str:
    return lib().fde_status_string(int(status)).decode()


def _check(status: int, what: str):
    if status != OK:
        raise FdeError(status, what)


def _ptr(t) -> int:
    if t is None:
        return 0
    if isinstance(t, int):
        return t
    return int(t.data_ptr())


def _stream(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def default_opts() -> FdeSolveOpts:
    o = FdeSolveOpts()
    lib().fde_default_opts(ctypes.byref(o))
    return o


def make_opts(method="gmres", restart=30, tol=1e-8, max_iters=5000, precision="f64", inner_tol=1e-4,
              max_outer=50, side="right", balance=False) -> FdeSolveOpts:
    o = FdeSolveOpts()
    o.method = {"pcg": PCG, "gmres": GMRES}[method] if isinstance(method, str) else method
    o.restart = restart
    o.tol = tol
    o.max_iters = max_iters
    o.precision = {"f64": PREC_F64, "f32": PREC_F32, "f32_ir": PREC_F32_IR}[precision] \
        if isinstance(precision, str) else precision
    o.inner_tol = inner_tol
    o.max_outer = max_outer
    o.side = {"right": SIDE_RIGHT, "left": SIDE_LEFT}[side] if isinstance(side, str) else side
    o.balance = int(bool(balance))
    return o


def make_problem(dim, n1, alpha, dt, n2=0, beta=0.0, len1=1.0, len2=1.0, scheme="ie", weights="gl1",
                 dp=None, dm=None, ep=None, em=None, dp_const=1.0, dm_const=1.0, ep_const=1.0,
                 em_const=1.0, tau_shift=False, order="tau_d") -> FdeProblem:
    """Problem struct; dp/dm/ep/em are device FP64 tensors (x fastest) or None."""
    p = FdeProblem()
    p.dim, p.n1, p.n2 = dim, n1, n2
    p.alpha, p.beta, p.len1, p.len2, p.dt = alpha, beta, len1, len2, dt
    p.scheme = {"ie": SCHEME_IMPLICIT_EULER, "cn": SCHEME_CRANK_NICOLSON}[scheme] if isinstance(scheme, str) else scheme
    p.weights = {"gl1": WEIGHTS_GL1, "wsgd2": WEIGHTS_WSGD2}[weights] if isinstance(weights, str) else weights
    p.dp, p.dm, p.ep, p.em = _ptr(dp) or None, _ptr(dm) or None, _ptr(ep) or None, _ptr(em) or None
    p.dp_const, p.dm_const, p.ep_const, p.em_const = dp_const, dm_const, ep_const, em_const
    p.tau_shift = int(bool(tau_shift))
    p.order = {"tau_d": ORDER_TAU_D, "d_tau": ORDER_D_TAU, "tau_df": ORDER_TAU_DF, "tri": ORDER_TRI}[order] \
        if isinstance(order, str) else order
    return p


def workspace_size(problem: FdeProblem, opts: FdeSolveOpts) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().fde_workspace_size(ctypes.byref(problem), ctypes.byref(opts), ctypes.byref(n)),
           "fde_workspace_size")
    return int(n.value)


def assemble_symbol(problem: FdeProblem, opts: FdeSolveOpts, workspace, nbytes: int, stream=None) -> int:
    h = ctypes.c_void_p(0)
    _check(lib().fde_assemble_symbol(ctypes.byref(problem), ctypes.byref(opts), _ptr(workspace), nbytes,
                                     ctypes.byref(h), _stream(stream)), "fde_assemble_symbol")
    return int(h.value)


def toeplitz_matvec(plan: int, dtype: int, x, y, stream=None):
    _check(lib().fde_toeplitz_matvec(plan, dtype, _ptr(x), _ptr(y), _stream(stream)), "fde_toeplitz_matvec")


def plan_set_schedule(plan: int, ctas: int, log_p1: int, stream=None):
    _check(lib().fde_plan_set_schedule(plan, ctas, log_p1, _stream(stream)), "fde_plan_set_schedule")


def autotune(plan: int, stream=None) -> tuple[int, int]:
    c, l = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().fde_autotune(plan, _stream(stream), ctypes.byref(c), ctypes.byref(l)), "fde_autotune")
    return c.value, l.value


MATVEC_NOALLOC_MAX_N = 4095


def toeplitz_matvec_noalloc(problem: FdeProblem, x, y, stream=None):
    """y = M x for a 1D problem without a plan or workspace (FP64, n1 <= 4095);
    the library's fixed static scratch holds the symbol data.  Calls that
    overlap in time on one device race on that scratch."""
    _check(lib().fde_toeplitz_matvec_noalloc(ctypes.byref(problem), _ptr(x), _ptr(y), _stream(stream)),
           "fde_toeplitz_matvec_noalloc")


def tau_solve(plan: int, dtype: int, r, z, stream=None):
    _check(lib().fde_tau_solve(plan, dtype, _ptr(r), _ptr(z), _stream(stream)), "fde_tau_solve")


def krylov_solve(plans: Sequence[int], b: Sequence, x: Sequence, opts: FdeSolveOpts, info_dev,
                 stream=None) -> int:
    """Launch one batched solve; returns the launch status (per-solve results land in info_dev)."""
    n = len(plans)
    arr = ctypes.c_void_p * n
    st = lib().fde_krylov_solve(arr(*plans), n, arr(*[_ptr(v) for v in b]), arr(*[_ptr(v) for v in x]),
                                ctypes.byref(opts), _ptr(info_dev), _stream(stream))
    _check(st, "fde_krylov_solve")
    return st


def step_rhs(plan: int, u_prev, f, b, stream=None):
    _check(lib().fde_step_rhs(plan, _ptr(u_prev), _ptr(f), _ptr(b), _stream(stream)), "fde_step_rhs")


def plan_scalars(plan: int) -> tuple[float, float, float]:
    c0, sr, ha = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().fde_plan_scalars(plan, ctypes.byref(c0), ctypes.byref(sr), ctypes.byref(ha)),
           "fde_plan_scalars")
    return c0.value, sr.value, ha.value


def measure_fp64_rate(stream=None) -> float:
    """FP64 FMA rate of the current device in TFLOP/s (fde_measure_fp64_rate)."""
    v = ctypes.c_double(0.0)
    _check(lib().fde_measure_fp64_rate(ctypes.byref(v), _stream(stream)), "fde_measure_fp64_rate")
    return v.value


def plan_destroy(plan: int):
    if plan:
        lib().fde_plan_destroy(plan)


def decode_info(raw: bytes, count: int) -> list[dict]:
    arr = (FdeSolveInfo * count).from_buffer_copy(raw)
    return [dict(status=a.status, iterations=a.iterations, outer=a.outer, restarts=a.restarts,
                 relres=a.relres, relres_est=a.relres_est, basis_sum=a.basis_sum, reorth=a.reorth,
                 cycles=a.cycles, residuals64=a.residuals64, iterations64=a.iterations64) for a in arr]


from .solver import Plan, solve_batch  # noqa: E402,F401
