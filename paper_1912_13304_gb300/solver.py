"""A plan object over the C ABI: owns the torch device buffers a plan needs
(workspace, coefficient arrays) and marshals calls.  No arithmetic of the
method happens here."""

from __future__ import annotations

from typing import Optional, Sequence

from . import (F32, F64, INFO_BYTES, assemble_symbol, autotune, decode_info, krylov_solve, make_opts, make_problem,
               plan_destroy, plan_scalars, plan_set_schedule, step_rhs, tau_solve, toeplitz_matvec, workspace_size)


def _torch():
    import torch
    return torch


class Plan:
    """An assembled plan (fde_assemble_symbol) plus the buffers it references."""

    def __init__(self, dim: int, n1: int, alpha: float, dt: float, *, n2: int = 0, beta: float = 0.0,
                 len1: float = 1.0, len2: float = 1.0, scheme: str = "ie", weights: str = "gl1",
                 dp=None, dm=None, ep=None, em=None, dp_const: float = 1.0, dm_const: float = 1.0,
                 ep_const: float = 1.0, em_const: float = 1.0, tau_shift: bool = False,
                 order: str = "tau_d", method: str = "gmres", restart: int = 30, precision: str = "f64",
                 device="cuda", stream=None, workspace_fill: Optional[int] = None):
        torch = _torch()
        self.device = torch.device(device)
        self._keep = []

        def dev(a, like=None):
            if a is None:
                return None
            if like is not None and a is like[0]:
                return like[1]
            t = torch.as_tensor(a, dtype=torch.float64).to(self.device).contiguous().reshape(-1)
            self._keep.append(t)
            return t

        dpt = dev(dp)
        dmt = dev(dm, like=(dp, dpt))
        ept = dev(ep)
        emt = dev(em, like=(ep, ept))
        self.dim, self.n1, self.n2 = dim, n1, (n2 if dim == 2 else 1)
        self.N = n1 * self.n2
        self.problem = make_problem(dim, n1, alpha, dt, n2=n2, beta=beta, len1=len1, len2=len2, scheme=scheme,
                                    weights=weights, dp=dpt, dm=dmt, ep=ept, em=emt, dp_const=dp_const,
                                    dm_const=dm_const, ep_const=ep_const, em_const=em_const,
                                    tau_shift=tau_shift, order=order)
        self.opts = make_opts(method=method, restart=restart, precision=precision)
        self.nbytes = workspace_size(self.problem, self.opts)
        self.workspace = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=self.device)
        if workspace_fill is not None:          # e.g. 0xFF: every double and float of it reads as NaN
            self.workspace.fill_(workspace_fill)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) & ~255
        self.handle = assemble_symbol(self.problem, self.opts, self._ws_ptr, self.nbytes, stream)
        self.c0, self.sr, self.h_alpha = plan_scalars(self.handle)

    @classmethod
    def from_workload(cls, w: dict, method: Optional[str] = None, precision: str = "f64", restart: Optional[int] = None,
                      order: Optional[str] = None, shift: Optional[bool] = None, device="cuda", stream=None,
                      workspace_fill: Optional[int] = None) -> "Plan":
        """Plan for one workload dict of ``workloads`` (coefficients as constants when they are)."""
        kw = dict(dim=w["dim"], n1=w["n1"], alpha=w["alpha"], dt=w["dt"], len1=w["length"], len2=w["length"],
                  weights=w["scheme"], tau_shift=w["shift"] if shift is None else shift,
                  order=w["order"] if order is None else order, method=method or w["method"],
                  restart=restart or max(1, w["restart"]), precision=precision, device=device, stream=stream,
                  workspace_fill=workspace_fill)
        if w["dim"] == 2:
            kw.update(n2=w["n2"], beta=w["beta"])
        if w["const_coeffs"]:
            kw.update(dp_const=float(w["dp"].reshape(-1)[0]), dm_const=float(w["dm"].reshape(-1)[0]))
            if w["dim"] == 2:
                kw.update(ep_const=float(w["ep"].reshape(-1)[0]), em_const=float(w["em"].reshape(-1)[0]))
        else:
            kw.update(dp=w["dp"].reshape(-1), dm=w["dm"].reshape(-1))
            if w["dim"] == 2:
                kw.update(ep=w["ep"].reshape(-1), em=w["em"].reshape(-1))
        return cls(**kw)

    def reassemble(self, stream=None):
        """Rebuild the plan's symbol data in its workspace on the stream
        (fde_assemble_symbol again with the same problem and options) and
        replace the host plan; the schedule returns to the default."""
        h = assemble_symbol(self.problem, self.opts, self._ws_ptr, self.nbytes, stream)
        plan_destroy(self.handle)
        self.handle = h

    # -- operators ---------------------------------------------------------
    def matvec(self, x, y=None, stream=None):
        torch = _torch()
        y = torch.empty_like(x) if y is None else y
        toeplitz_matvec(self.handle, F64 if x.dtype == torch.float64 else F32, x, y, stream)
        return y

    def tau(self, r, z=None, stream=None):
        torch = _torch()
        z = torch.empty_like(r) if z is None else z
        tau_solve(self.handle, F64 if r.dtype == torch.float64 else F32, r, z, stream)
        return z

    def rhs(self, u_prev, f=None, b=None, stream=None):
        torch = _torch()
        b = torch.empty_like(u_prev) if b is None else b
        step_rhs(self.handle, u_prev, f, b, stream)
        return b

    def solve(self, b, x=None, **kw) -> dict:
        torch = _torch()
        x = torch.zeros_like(b) if x is None else x
        info = solve_batch([self], [b], [x], **kw)[0]
        info["x"] = x
        return info

    def set_schedule(self, ctas: int = 0, log_p1: int = 0, stream=None):
        """Fix the transform schedule (fde_plan_set_schedule)."""
        plan_set_schedule(self.handle, ctas, log_p1, stream)

    def autotune(self, stream=None) -> tuple[int, int]:
        """Time the feasible schedules and keep the fastest (fde_autotune):
        returns (ctas, log_p1)."""
        return autotune(self.handle, stream)

    def close(self):
        if getattr(self, "handle", 0):
            plan_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_SIDE_STREAMS: dict = {}


def reassemble_all(plans: Sequence[Plan], streams: int = 16) -> None:
    """Rebuild every plan's symbol data (fde_assemble_symbol again), the plans
    spread round-robin over `streams` side streams that start after, and
    join, the current stream.  One plan's assembly kernels are single-CTA
    jobs, so plans on different streams assemble on different SMs at once
    instead of one after another."""
    torch = _torch()
    if not plans:
        return
    dev = torch.cuda.current_device()
    pool = _SIDE_STREAMS.setdefault(dev, [])
    k = max(1, min(streams, len(plans)))
    while len(pool) < k:
        pool.append(torch.cuda.Stream(device=dev))
    cur = torch.cuda.current_stream()
    start = torch.cuda.Event()
    start.record(cur)
    for st in pool[:k]:
        st.wait_event(start)
    for i, p in enumerate(plans):
        p.reassemble(stream=pool[i % k])
    for st in pool[:k]:
        done = torch.cuda.Event()
        done.record(st)
        cur.wait_event(done)


def solve_batch(plans: Sequence[Plan], b: Sequence, x: Sequence, tol: float = 1e-8, max_iters: int = 5000,
                inner_tol: float = 1e-4, max_outer: int = 50, side: str = "right", info_dev=None, stream=None,
                read_info: bool = True, balance: bool = False):
    """One fde_krylov_solve launch over several plans (same method/precision/restart).
    With ``balance``, ``info_dev`` must hold the previous solve's results for
    the same plans (or zeros): team sizes follow its iteration counts."""
    torch = _torch()
    p0 = plans[0]
    opts = make_opts(method=p0.opts.method, restart=p0.opts.restart, tol=tol, max_iters=max_iters,
                     precision=p0.opts.precision, inner_tol=inner_tol, max_outer=max_outer, side=side,
                     balance=balance)
    if info_dev is None:
        info_dev = torch.zeros(len(plans) * INFO_BYTES, dtype=torch.uint8, device=p0.device)
    krylov_solve([p.handle for p in plans], b, x, opts, info_dev, stream)
    if not read_info:
        return info_dev
    raw = info_dev.cpu().numpy().tobytes()
    return decode_info(raw, len(plans))


class TimeStepper:
    """Implicit-Euler time stepping of several plans together (Sec. 1.2: each
    step solves M u_m = c0 u_{m-1} + h^alpha f with x0 = u_{m-1}): per step one
    fde_step_rhs per plan and one batched fde_krylov_solve.  With ``graph``
    the whole loop of ``steps`` steps is captured once in a CUDA graph and
    ``run()`` replays it; ``u`` (device tensors, updated in place) and the
    per-step info buffer are the graph's fixed inputs and outputs.  With
    ``balance`` each step sizes the instances' teams from the previous step's
    iteration counts (the first step splits evenly)."""

    def __init__(self, plans: Sequence[Plan], u: Sequence, steps: int, *, tol: float = 1e-8,
                 max_iters: int = 5000, inner_tol: float = 1e-4, max_outer: int = 50, balance: bool = True,
                 graph: bool = True):
        torch = _torch()
        self.plans = list(plans)
        self.u = list(u)
        self.steps = steps
        self.b = [torch.empty_like(x) for x in self.u]
        self.isz = len(self.plans) * INFO_BYTES
        self.info = torch.zeros(steps * self.isz, dtype=torch.uint8, device=self.u[0].device)
        self.kw = dict(tol=tol, max_iters=max_iters, inner_tol=inner_tol, max_outer=max_outer, balance=balance)
        self.graph = None
        if graph:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self._loop()
            self.graph = g

    def _loop(self, events=None):
        for m in range(self.steps):
            for k, p in enumerate(self.plans):
                p.rhs(self.u[k], b=self.b[k])
            cur = self.info[m * self.isz:(m + 1) * self.isz]
            if self.kw["balance"]:
                if m == 0:
                    cur.zero_()
                else:
                    cur.copy_(self.info[(m - 1) * self.isz:m * self.isz])
            if events is not None:
                events[m][0].record()
            solve_batch(self.plans, self.b, self.u, info_dev=cur, read_info=False, **self.kw)
            if events is not None:
                events[m][1].record()

    def run_eager(self, events=None):
        """All steps as eager launches; events[m] = (start, end) CUDA events
        recorded around step m's solve launch."""
        self._loop(events)

    def run(self):
        """All steps on the current stream (graph replay or eager launches)."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self._loop()

    def infos(self) -> list[list[dict]]:
        """Per step, per plan: the decoded fde_solve_info."""
        flat = decode_info(self.info.cpu().numpy().tobytes(), self.steps * len(self.plans))
        n = len(self.plans)
        return [flat[m * n:(m + 1) * n] for m in range(self.steps)]
