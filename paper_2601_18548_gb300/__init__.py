"""GB300-native neural GCDF hot path (arXiv 2601.18548).

Python binding of libgcdf: the functions below have the names of the C entry
points in include/gcdf.h and only marshal arguments (PyTorch tensors -> device
pointers, the current CUDA stream).  Every step of the computation runs in the
library's CUDA kernels; if the library is not built, the first call raises.

    net = create_net(n_dof=9, hidden=256, n_layers=4, weights=w, precision="bf16")
    f, g = query(net, q, p)                       # per-pair f and df/dq (Eq. 14, 15)
    c, g, a = collision_cost(net, q, p, "softmin", 0.02)
    q_opt, merit, acc = plan_solve(net, [problem, ...], PlanParams())   # Sec. IV-A optimiser
    server = Server(budget_bytes, max_active, max_queued, PlanParams())  # continuous batching
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import GcdfError  # noqa: F401

_PREC = {"fp32": _lib.GCDF_FP32, "bf16": _lib.GCDF_BF16, "fp16": _lib.GCDF_FP16, "fp8": _lib.GCDF_FP8}
_RED = {"min": _lib.GCDF_RED_MIN, "softmin": _lib.GCDF_RED_SOFTMIN, "hinge": _lib.GCDF_RED_HINGE}


def _desc(n_dof, hidden, n_layers, precision):
    return _lib.NetDesc(int(n_dof), int(hidden), int(n_layers), _PREC[precision])


def weight_count(n_dof: int, hidden: int, n_layers: int) -> int:
    d = _desc(n_dof, hidden, n_layers, "fp32")
    return int(_lib.load().gcdf_weight_count(ctypes.byref(d)))


class Net:
    """Owner of a gcdf_net handle (device weights on the current device)."""

    def __init__(self, handle, n_dof, hidden, n_layers, precision):
        self.handle = handle
        self.n_dof, self.hidden, self.n_layers, self.precision = n_dof, hidden, n_layers, precision

    def __del__(self):
        destroy_net(self)


def create_net(n_dof: int, hidden: int, n_layers: int, weights, precision: str = "fp32") -> Net:
    """gcdf_create_net: weights is a flat FP32 host array (numpy or CPU tensor)."""
    lib = _lib.load()
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32))
    d = _desc(n_dof, hidden, n_layers, precision)
    out = ctypes.c_void_p()
    _lib.check(lib.gcdf_create_net(ctypes.byref(d), w.ctypes.data, w.size, ctypes.byref(out)))
    return Net(out, n_dof, hidden, n_layers, precision)


def destroy_net(net: Net) -> None:
    """gcdf_destroy_net."""
    if getattr(net, "handle", None) and net.handle.value:
        _lib.load().gcdf_destroy_net(net.handle)
        net.handle = ctypes.c_void_p()


def _ptr(t, dtype=torch.float32, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def query(net: Net, q: torch.Tensor, p: torch.Tensor, part_offsets=None, part_idx=None,
          shift=None, with_grad: bool = True, out=None, stream=None):
    """gcdf_query: per-pair f (P,) and df/dq (P, n) in stacked order (Eq. 14)."""
    lib = _lib.load()
    N, M = q.shape[0], p.shape[0]
    P = N * M if part_offsets is None else int(part_idx.numel())
    if out is None:
        f = torch.empty(P, device=q.device, dtype=torch.float32)
        g = torch.empty(P, net.n_dof, device=q.device, dtype=torch.float32) if with_grad else None
    else:
        f, g = out
    _lib.check(lib.gcdf_query(net.handle, _ptr(q, name="q"), N, _ptr(p, name="p"), M,
                              _ptr(part_offsets, torch.int32, "part_offsets"),
                              _ptr(part_idx, torch.int32, "part_idx"), P,
                              _ptr(shift, name="shift"), _ptr(f, name="f"),
                              _ptr(g, name="grad"), _stream(stream)))
    return f, g


def collision_cost(net: Net, q: torch.Tensor, p: torch.Tensor, reduction: str = "softmin",
                   param: float = 0.02, part_offsets=None, part_idx=None, shift=None,
                   out=None, stream=None):
    """gcdf_collision_cost: per-waypoint cost (N,), grad (N, n), argmin (N,)."""
    lib = _lib.load()
    N, M = q.shape[0], p.shape[0]
    P = N * M if part_offsets is None else int(part_idx.numel())
    if out is None:
        cost = torch.empty(N, device=q.device, dtype=torch.float32)
        grad = torch.empty(N, net.n_dof, device=q.device, dtype=torch.float32)
        amin = torch.empty(N, device=q.device, dtype=torch.int32)
    else:
        cost, grad, amin = out
    _lib.check(lib.gcdf_collision_cost(net.handle, _ptr(q, name="q"), N, _ptr(p, name="p"), M,
                                       _ptr(part_offsets, torch.int32, "part_offsets"),
                                       _ptr(part_idx, torch.int32, "part_idx"), P,
                                       _ptr(shift, name="shift"), _RED[reduction], float(param),
                                       _ptr(cost, name="cost"), _ptr(grad, name="grad"),
                                       _ptr(amin, torch.int32, "argmin"), _stream(stream)))
    return cost, grad, amin


def collision_cost_noalloc(net: Net, q: torch.Tensor, p: torch.Tensor, reduction: str = "softmin",
                           param: float = 0.02, part_offsets=None, part_idx=None, shift=None,
                           out=None, stream=None):
    """gcdf_collision_cost_noalloc: as collision_cost, but the library allocates
    nothing (its temporaries live in a fixed per-device array).  For callers that
    must not allocate once running; pass preallocated `out` tensors as well."""
    lib = _lib.load()
    N, M = q.shape[0], p.shape[0]
    P = N * M if part_offsets is None else int(part_idx.numel())
    if out is None:
        cost = torch.empty(N, device=q.device, dtype=torch.float32)
        grad = torch.empty(N, net.n_dof, device=q.device, dtype=torch.float32)
        amin = torch.empty(N, device=q.device, dtype=torch.int32)
    else:
        cost, grad, amin = out
    _lib.check(lib.gcdf_collision_cost_noalloc(net.handle, _ptr(q, name="q"), N, _ptr(p, name="p"), M,
                                               _ptr(part_offsets, torch.int32, "part_offsets"),
                                               _ptr(part_idx, torch.int32, "part_idx"), P,
                                               _ptr(shift, name="shift"), _RED[reduction], float(param),
                                               _ptr(cost, name="cost"), _ptr(grad, name="grad"),
                                               _ptr(amin, torch.int32, "argmin"), _stream(stream)))
    return cost, grad, amin


def project(net: Net, q: torch.Tensor, p: torch.Tensor, part_offsets=None, part_idx=None, shift=None,
            m_diag=None, out=None, stream=None):
    """gcdf_project: q_z = q - f M^{-1} df/dq for every pair (Theorem 1), (P, n)."""
    lib = _lib.load()
    N, M = q.shape[0], p.shape[0]
    P = N * M if part_offsets is None else int(part_idx.numel())
    qz = torch.empty(P, net.n_dof, device=q.device, dtype=torch.float32) if out is None else out
    _lib.check(lib.gcdf_project(net.handle, _ptr(q, name="q"), N, _ptr(p, name="p"), M,
                                _ptr(part_offsets, torch.int32, "part_offsets"),
                                _ptr(part_idx, torch.int32, "part_idx"), P, _ptr(shift, name="shift"),
                                _ptr(m_diag, name="m_diag"), _ptr(qz, name="q_out"), _stream(stream)))
    return qz


def partition(base_xy: torch.Tensor, p: torch.Tensor, radius: float, stream=None):
    """gcdf_partition_offsets + gcdf_partition_indices: CSR lists (offsets
    (N+1,) int32, idx int32) of the points within planar range `radius` of
    every waypoint's base position (Sec. IV-A).  Reads the list length back
    (one synchronisation) to size idx."""
    lib = _lib.load()
    N, M = base_xy.shape[0], p.shape[0]
    off = torch.empty(N + 1, device=p.device, dtype=torch.int32)
    bp, pp = _ptr(base_xy, name="base_xy"), _ptr(p, name="p")
    _lib.check(lib.gcdf_partition_offsets(bp, N, pp, M, float(radius), _ptr(off, torch.int32, "offsets"),
                                          _stream(stream)))
    total = int(off[-1].item())
    idx = torch.empty(max(total, 4), device=p.device, dtype=torch.int32)
    _lib.check(lib.gcdf_partition_indices(bp, N, pp, M, float(radius), _ptr(off, torch.int32, "offsets"),
                                          _ptr(idx, torch.int32, "idx"), _stream(stream)))
    return off, idx[:total]


def jacobian_scatter(grad: torch.Tensor, n_waypoints: int, part_offsets=None, n_points: int = 0,
                     with_values: bool = True, stream=None):
    """gcdf_jacobian_scatter: CSR (row_ptr int64, col_idx int32, values) of the
    (P x 2Nn) Jacobian of Eq. (17) from the dense (P, n) block."""
    lib = _lib.load()
    P, n = grad.shape
    row_ptr = torch.empty(P + 1, device=grad.device, dtype=torch.int64)
    col = torch.empty(max(P * n, 4), device=grad.device, dtype=torch.int32)
    val = torch.empty(max(P * n, 4), device=grad.device, dtype=torch.float32) if with_values else None
    _lib.check(lib.gcdf_jacobian_scatter(_ptr(grad, name="grad"), int(n_waypoints), n,
                                         _ptr(part_offsets, torch.int32, "part_offsets"), int(n_points), P,
                                         _ptr(row_ptr, torch.int64, "row_ptr"), _ptr(col, torch.int32, "col_idx"),
                                         None if val is None else _ptr(val, name="values"), _stream(stream)))
    return row_ptr, col[: P * n], (None if val is None else val[: P * n])


def device_status(net: Net) -> int:
    """gcdf_device_status: 0, or the bits of a bounded device wait that gave up."""
    v = ctypes.c_int(0)
    _lib.check(_lib.load().gcdf_device_status(net.handle, ctypes.byref(v)))
    return v.value


def set_profile_events(net: Net, start=None, stop=None) -> None:
    """gcdf_set_profile_events: torch.cuda.Event pair (enable_timing=True) or None."""
    a = None if start is None else ctypes.c_void_p(start.cuda_event)
    b = None if stop is None else ctypes.c_void_p(stop.cuda_event)
    _lib.check(_lib.load().gcdf_set_profile_events(net.handle, a, b))


def set_active_set(net: Net, enable: bool) -> None:
    """gcdf_set_active_set: HINGE / MIN in two passes (values, then the active
    pairs' gradients) when enabled (the default), in one pass otherwise."""
    _lib.check(_lib.load().gcdf_set_active_set(net.handle, 1 if enable else 0))


def selftest_wait_expiry(net: Net, limit_cycles: int = 200000):
    """gcdf_selftest_wait_expiry: [producer wait expired, epilogue wait expired,
    abort flag raised] of a probe whose waits can never complete."""
    seen = (ctypes.c_int * 3)()
    _lib.check(_lib.load().gcdf_selftest_wait_expiry(net.handle, int(limit_cycles), seen))
    return [int(x) for x in seen]


def diag_fp32_fma(blocks: int, threads: int, iters: int, sink: torch.Tensor, stream=None) -> int:
    """gcdf_diag_fp32_fma: enqueue the FMA-rate loop; returns its FLOP count."""
    r = _lib.load().gcdf_diag_fp32_fma(int(blocks), int(threads), int(iters), _ptr(sink, name="sink"),
                                       _stream(stream))
    if r < 0:
        _lib.check(int(-r))
    return int(r)


def release_cached_memory() -> None:
    """gcdf_release_cached_memory: trim the library's temporary-memory pool."""
    _lib.check(_lib.load().gcdf_release_cached_memory())


def last_error() -> str:
    """gcdf_last_error."""
    m = _lib.load().gcdf_last_error()
    return m.decode() if m else ""


# ---------------------------------------------------------------------------
# Trajectory optimisation (gcdf_plan_solve) and the planning server
# ---------------------------------------------------------------------------

class PlanParams:
    """gcdf_plan_params: cost weights, margin, damping and step count."""

    def __init__(self, dt=0.1, w_trans=1.0, w_rot=0.5, w_goal=100.0, mu=1.0, delta=0.05,
                 lambda0=1.0, lambda_min=1e-6, lambda_max=1e8, iterations=50, partition_radius=0.0):
        self.dt, self.w_trans, self.w_rot, self.w_goal = dt, w_trans, w_rot, w_goal
        self.mu, self.delta, self.iterations = mu, delta, iterations
        self.lambda0, self.lambda_min, self.lambda_max = lambda0, lambda_min, lambda_max
        self.partition_radius = partition_radius

    def c(self):
        return _lib.PlanParams(self.dt, self.w_trans, self.w_rot, self.w_goal, self.mu, self.delta,
                               self.lambda0, self.lambda_min, self.lambda_max, int(self.iterations),
                               float(self.partition_radius))


def plan_solve(net: Net, problems, params: PlanParams, history: bool = True, stream=None):
    """gcdf_plan_solve.  problems: list of dicts with CUDA tensors q_start (n,),
    q_goal (n,), points (M, 3) and optional q_init (N, n), plus n_waypoints.
    Returns q (sum N, n) and, with history, merit (R, iters + 1) FP64 and
    accepted (R, iters + 1) uint8."""
    lib = _lib.load()
    R = len(problems)
    arr = (_lib.PlanProblem * max(R, 1))()
    rows = 0
    for r, pr in enumerate(problems):
        pts = pr["points"]
        arr[r] = _lib.PlanProblem(int(pr["n_waypoints"]), _ptr(pr["q_start"], name="q_start"),
                                  _ptr(pr["q_goal"], name="q_goal"), _ptr(pr.get("q_init"), name="q_init"),
                                  _ptr(pts, name="points") if pts.shape[0] > 0 else None, int(pts.shape[0]))
        rows += int(pr["n_waypoints"])
    dev = problems[0]["q_start"].device if R else torch.device("cuda")
    q = torch.empty(rows, net.n_dof, device=dev, dtype=torch.float32)
    merit = acc = None
    if history:
        merit = torch.empty(R, params.iterations + 1, device=dev, dtype=torch.float64)
        acc = torch.empty(R, params.iterations + 1, device=dev, dtype=torch.uint8)
    prm = params.c()
    _lib.check(lib.gcdf_plan_solve(net.handle, arr, R, ctypes.byref(prm), _ptr(q, name="q_out"),
                                   None if merit is None else merit.data_ptr(),
                                   None if acc is None else acc.data_ptr(), _stream(stream)))
    return q, merit, acc


def plan_request_bytes(net: Net, n_waypoints: int, n_points: int) -> int:
    """gcdf_plan_request_bytes: what one request counts against a server's budget."""
    return int(_lib.load().gcdf_plan_request_bytes(net.handle, int(n_waypoints), int(n_points)))


class Server:
    """gcdf_server_*: planning requests in, optimised trajectories out, with
    continuous batching on the device that is current at construction."""

    def __init__(self, budget_bytes: int, max_active: int, max_queued: int, params: PlanParams):
        self._lib = _lib.load()
        d = _lib.ServerDesc(int(budget_bytes), int(max_active), int(max_queued), params.c())
        h = ctypes.c_void_p()
        _lib.check(self._lib.gcdf_server_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        self._shapes = {}

    def submit(self, net: Net, n_waypoints: int, q_start, q_goal, points) -> int:
        """gcdf_plan_submit with host arrays; returns the ticket, or raises
        GcdfError with code GCDF_EAGAIN when the queue is full."""
        qs = np.ascontiguousarray(np.asarray(q_start, dtype=np.float32))
        qg = np.ascontiguousarray(np.asarray(q_goal, dtype=np.float32))
        pts = np.ascontiguousarray(np.asarray(points, dtype=np.float32).reshape(-1, 3))
        rq = _lib.PlanRequest(net.handle, int(n_waypoints), qs.ctypes.data, qg.ctypes.data,
                              pts.ctypes.data if pts.shape[0] else None, int(pts.shape[0]))
        t = ctypes.c_uint64(0)
        _lib.check(self._lib.gcdf_plan_submit(self.handle, ctypes.byref(rq), ctypes.byref(t)))
        self._shapes[t.value] = (int(n_waypoints), net.n_dof)
        return t.value

    def poll(self, ticket: int):
        """gcdf_plan_poll: None while pending, else a dict with q (N, n),
        merit, accepted_steps and the server-clock times."""
        N, n = self._shapes[ticket]
        q = np.empty((N, n), dtype=np.float32)
        res = _lib.PlanResult(q.ctypes.data, 0.0, 0, 0.0, 0.0, 0.0)
        rc = self._lib.gcdf_plan_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(res))
        if rc == _lib.GCDF_PENDING:
            return None
        _lib.check(rc)
        del self._shapes[ticket]
        return {"q": q, "merit": res.merit, "accepted_steps": res.accepted_steps,
                "submit_s": res.submit_s, "admit_s": res.admit_s, "done_s": res.done_s}

    def clock(self) -> float:
        return float(self._lib.gcdf_server_clock(self.handle))

    def stats(self) -> dict:
        """gcdf_server_stats_get: the worker loop's step counters."""
        st = _lib.ServerStats()
        _lib.check(self._lib.gcdf_server_stats_get(self.handle, ctypes.byref(st)))
        return {"steps": int(st.steps), "step_device_s": st.step_device_s, "step_host_s": st.step_host_s,
                "pass_s": st.pass_s, "active_sum": int(st.active_sum)}

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            self._lib.gcdf_server_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        self.close()


# ---------------------------------------------------------------------------
# Differentiable fit (gcdf_fit_forward / gcdf_fit_vjp / gcdf_fit_value_grad /
# gcdf_fit_vjp2); precision "fp32" (SIMT GEMMs) or "bf16" (tensor-core GEMMs,
# BF16 operands, FP32 accumulation and master weights)
# ---------------------------------------------------------------------------

def _fit_desc(shape, precision):
    if precision not in ("fp32", "bf16"):
        raise ValueError(f"fit precision {precision!r}: 'fp32' or 'bf16'")
    return _lib.FitDesc(*[int(x) for x in shape], _PREC[precision])


def fit_forward(shape, weights: torch.Tensor, q: torch.Tensor, p: torch.Tensor, stream=None,
                precision="fp32") -> torch.Tensor:
    """gcdf_fit_forward: f (B,) per sample; shape = (n_dof, hidden, n_layers)."""
    d = _fit_desc(shape, precision)
    f = torch.empty(q.shape[0], device=q.device, dtype=torch.float32)
    _lib.check(_lib.load().gcdf_fit_forward(ctypes.byref(d), _ptr(weights, name="weights"), _ptr(q, name="q"),
                                            _ptr(p, name="p"), int(q.shape[0]), _ptr(f, name="f"), _stream(stream)))
    return f


def fit_vjp(shape, weights, q, p, g_f, want_dq=True, stream=None, precision="fp32"):
    """gcdf_fit_vjp: (dweights, dq or None) for the upstream gradient g_f (B,)."""
    d = _fit_desc(shape, precision)
    dw = torch.empty_like(weights)
    dq = torch.empty_like(q) if want_dq else None
    _lib.check(_lib.load().gcdf_fit_vjp(ctypes.byref(d), _ptr(weights, name="weights"), _ptr(q, name="q"),
                                        _ptr(p, name="p"), int(q.shape[0]), _ptr(g_f.contiguous(), name="g_f"),
                                        _ptr(dw, name="dweights"), None if dq is None else _ptr(dq, name="dq"),
                                        _stream(stream)))
    return dw, dq


def fit_value_grad(shape, weights, q, p, stream=None, precision="fp32"):
    """gcdf_fit_value_grad: (f (B,), grad_q f (B, n)) per sample."""
    d = _fit_desc(shape, precision)
    f = torch.empty(q.shape[0], device=q.device, dtype=torch.float32)
    dq = torch.empty_like(q)
    _lib.check(_lib.load().gcdf_fit_value_grad(ctypes.byref(d), _ptr(weights, name="weights"), _ptr(q, name="q"),
                                               _ptr(p, name="p"), int(q.shape[0]), _ptr(f, name="f"),
                                               _ptr(dq, name="dq"), _stream(stream)))
    return f, dq


def fit_vjp2(shape, weights, q, p, g_f, G_q, stream=None, precision="fp32"):
    """gcdf_fit_vjp2: dweights of sum_b g_b f_b + G_b . grad_q f_b."""
    d = _fit_desc(shape, precision)
    dw = torch.empty_like(weights)
    _lib.check(_lib.load().gcdf_fit_vjp2(ctypes.byref(d), _ptr(weights, name="weights"), _ptr(q, name="q"),
                                         _ptr(p, name="p"), int(q.shape[0]), _ptr(g_f.contiguous(), name="g_f"),
                                         _ptr(G_q.contiguous(), name="G_q"), _ptr(dw, name="dweights"),
                                         _stream(stream)))
    return dw


def fit_tape_bytes(shape, batch: int, precision="bf16") -> int:
    """gcdf_fit_tape_bytes: device bytes of the tape of a BF16 forward pass."""
    d = _fit_desc(shape, precision)
    n = ctypes.c_size_t(0)
    _lib.check(_lib.load().gcdf_fit_tape_bytes(ctypes.byref(d), int(batch), ctypes.byref(n)))
    return int(n.value)


def fit_forward_tape(shape, weights, q, p, stream=None, precision="bf16"):
    """gcdf_fit_forward_tape: (f (B,), tape) — the tape (a uint8 CUDA tensor)
    holds what fit_vjp_tape needs for the same weights, q and p."""
    d = _fit_desc(shape, precision)
    B = int(q.shape[0])
    f = torch.empty(B, device=q.device, dtype=torch.float32)
    tape = torch.empty(max(fit_tape_bytes(shape, B, precision), 1), device=q.device, dtype=torch.uint8)
    _lib.check(_lib.load().gcdf_fit_forward_tape(ctypes.byref(d), _ptr(weights, name="weights"), _ptr(q, name="q"),
                                                 _ptr(p, name="p"), B, _ptr(f, name="f"), _ptr(tape, torch.uint8, name="tape"),
                                                 tape.numel(), _stream(stream)))
    return f, tape


def fit_vjp_tape(shape, weights, q, p, g_f, tape, want_dq=True, stream=None, precision="bf16"):
    """gcdf_fit_vjp_tape: fit_vjp from the tape of fit_forward_tape (same
    weights, q and p), without repeating the forward pass."""
    d = _fit_desc(shape, precision)
    dw = torch.empty_like(weights)
    dq = torch.empty_like(q) if want_dq else None
    _lib.check(_lib.load().gcdf_fit_vjp_tape(ctypes.byref(d), _ptr(weights, name="weights"), _ptr(q, name="q"),
                                             _ptr(p, name="p"), int(q.shape[0]), _ptr(g_f.contiguous(), name="g_f"),
                                             _ptr(tape, torch.uint8, name="tape"), tape.numel(), _ptr(dw, name="dweights"),
                                             None if dq is None else _ptr(dq, name="dq"), _stream(stream)))
    return dw, dq


def fit_device_status() -> int:
    """gcdf_fit_device_status: synchronise; the fit kernels' status word since
    the last call (0 = every tensor-core wait completed), then clear it."""
    v = ctypes.c_int(0)
    _lib.check(_lib.load().gcdf_fit_device_status(ctypes.byref(v)))
    return int(v.value)


class FieldFunction(torch.autograd.Function):
    """f(q_b, p_b; weights) as an autograd.Function: the forward and both
    vector-Jacobian products (weights and q) run in libgcdf's kernels.  With
    BF16 products the forward keeps its tape for the backward (autograd's
    version check on the saved weights and q guards against in-place changes
    in between); with FP32 the backward recomputes the forward."""

    @staticmethod
    def forward(ctx, weights, q, p, shape, precision):
        ctx.save_for_backward(weights, q, p)
        ctx.shape, ctx.precision = shape, precision
        if precision == "bf16":
            f, ctx.tape = fit_forward_tape(shape, weights.detach(), q.detach(), p, precision=precision)
            return f
        ctx.tape = None
        return fit_forward(shape, weights.detach(), q.detach(), p, precision=precision)

    @staticmethod
    def backward(ctx, g_f):
        weights, q, p = ctx.saved_tensors
        if ctx.tape is not None:
            dw, dq = fit_vjp_tape(ctx.shape, weights.detach(), q.detach(), p, g_f.detach().float(), ctx.tape,
                                  want_dq=ctx.needs_input_grad[1], precision=ctx.precision)
            ctx.tape = None
        else:
            dw, dq = fit_vjp(ctx.shape, weights.detach(), q.detach(), p, g_f.detach().float(),
                             want_dq=ctx.needs_input_grad[1], precision=ctx.precision)
        return dw, dq, None, None, None


def field(weights: torch.Tensor, q: torch.Tensor, p: torch.Tensor, shape, precision="fp32") -> torch.Tensor:
    """Differentiable per-sample field values (weights: flat FP32 CUDA tensor)."""
    return FieldFunction.apply(weights, q, p, tuple(shape), precision)


class FieldGradFunction(torch.autograd.Function):
    """(f, grad_q f)(q_b, p_b; weights) as an autograd.Function for losses on
    the field and its gradient (the gradient, eikonal and tension terms of
    Table I); the backward pass is gcdf_fit_vjp2 and gives the weight gradient
    only."""

    @staticmethod
    def forward(ctx, weights, q, p, shape, precision):
        ctx.save_for_backward(weights, q, p)
        ctx.shape, ctx.precision = shape, precision
        return fit_value_grad(shape, weights.detach(), q.detach(), p, precision=precision)

    @staticmethod
    def backward(ctx, g_f, G_q):
        if ctx.needs_input_grad[1] or ctx.needs_input_grad[2]:
            raise RuntimeError("field_grad: gradients with respect to q or p are not provided")
        weights, q, p = ctx.saved_tensors
        if g_f is None:
            g_f = torch.zeros(q.shape[0], device=q.device, dtype=torch.float32)
        if G_q is None:
            G_q = torch.zeros_like(q)
        dw = fit_vjp2(ctx.shape, weights.detach(), q.detach(), p, g_f.detach().float(), G_q.detach().float(),
                      precision=ctx.precision)
        return dw, None, None, None, None


def field_grad(weights: torch.Tensor, q: torch.Tensor, p: torch.Tensor, shape, precision="fp32"):
    """Differentiable (f, grad_q f) per sample, with respect to the weights."""
    return FieldGradFunction.apply(weights, q, p, tuple(shape), precision)
