"""Python binding of the libsg C ABI (include/sg.h): argument marshalling only.

Device memory and streams come from PyTorch; every step of the method runs in
the library's CUDA kernels.  Importing this module loads the shared library
and fails loudly if it has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

# --------------------------------------------------------------- constants
SG_OK, SG_EINVAL, SG_ENOMEM, SG_ECUDA, SG_EUNSUPPORTED, SG_EFULL = 0, 1, 2, 3, 4, 5
PROBLEM_ATTITUDE, PROBLEM_LQ, PROBLEM_EXAMPLE3 = 0, 1, 2
# FP64; FP32 direction with an FP64 residual; FP32 direction with a pair-of-floats residual
PREC_FP64, PREC_MIXED, PREC_MIXED_PAIR = 0, 1, 2
CONVERGED, MAXITER, NONFINITE, SINGULAR, BADINPUT = 0, 1, 2, 3, 4
EVAL_FP64, EVAL_TF32X3, EVAL_DF32 = 0, 1, 2


class Problem(C.Structure):
    _fields_ = [("kind", C.c_int32), ("m", C.c_int32),
                ("J", C.c_double * 3), ("hmom", C.c_double * 3), ("B", C.c_double * 9),
                ("wv", C.c_double), ("ww", C.c_double), ("r", C.c_double),
                ("tv", C.c_double), ("tw", C.c_double),
                ("A", C.c_double * 36), ("Blq", C.c_double * 18), ("Q", C.c_double * 36),
                ("R", C.c_double * 9), ("QT", C.c_double * 36), ("d_target", C.c_void_p)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("precision", C.c_int32),
                ("damping", C.c_int32), ("persistent", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("graph", C.c_int32), ("warm_start", C.c_int32), ("cond_warps", C.c_int32)]


class SGError(RuntimeError):
    pass


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise SGError(f"libsg.so not built ({path}); run __graft_entry__.build() first")
    lib = C.CDLL(path)
    P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int, C.c_double
    lib.sg_last_error.restype = C.c_char_p
    lib.sg_build_grid.argtypes = [I32, I32, P, P, C.POINTER(P)]
    lib.sg_grid_info.argtypes = [P, C.POINTER(I64), C.POINTER(I32), C.POINTER(I32),
                                 C.POINTER(P), C.POINTER(P), C.POINTER(P)]
    lib.sg_grid_free.argtypes = [P]
    lib.sg_grid_free.restype = None
    lib.sg_solve_workspace_bytes.argtypes = [I64, I32, I32]
    lib.sg_solve_workspace_bytes.restype = C.c_size_t
    lib.sg_solve_bvps.argtypes = [C.POINTER(Problem), P, I64, P, P, I32, C.POINTER(SolveOpts),
                                  P, C.c_size_t, P, P, P, P, P, P, P]
    lib.sg_solve_bvps_static.argtypes = [C.POINTER(Problem), P, I64, P, P, I32, C.POINTER(SolveOpts),
                                         P, P, P, P, P, P, P]
    lib.sg_solve_bvps_static.restype = C.c_int
    lib.sg_autotune_solve.argtypes = [C.POINTER(Problem), P, I64, P, P, I32, C.POINTER(SolveOpts), P,
                                      C.c_size_t, P, P, P, P, P, C.POINTER(SolveOpts), C.POINTER(D), I32, P]
    lib.sg_autotune_solve.restype = C.c_int
    lib.sg_simulate_closed_loop.argtypes = [C.POINTER(Problem), P, P, I64, I32, D, I32, P, P, P, P, P]
    lib.sg_simulate_closed_loop.restype = C.c_int
    lib.sg_build_surpluses.argtypes = [P, P, I32, C.POINTER(P), P]
    lib.sg_surplus_info.argtypes = [P, C.POINTER(I64), C.POINTER(I32), C.POINTER(P)]
    lib.sg_surplus_free.argtypes = [P]
    lib.sg_surplus_free.restype = None
    lib.sg_eval_feedback.argtypes = [P, P, I64, I32, P, P]
    lib.sg_sincos_probe.argtypes = [P, I64, P, P, P]
    lib.sg_attitude_targets.argtypes = [C.POINTER(Problem), P, I64, P, P, P]
    lib.sg_attitude_targets.restype = C.c_int
    lib.sg_pool_workspace_bytes.argtypes = [I64, I32, I32]
    lib.sg_pool_workspace_bytes.restype = C.c_size_t
    lib.sg_pool_create.argtypes = [C.POINTER(Problem), I64, I32, C.POINTER(SolveOpts), P, C.c_size_t,
                                   C.POINTER(P), P]
    lib.sg_pool_free.argtypes = [P]
    lib.sg_pool_free.restype = None
    lib.sg_pool_info.argtypes = [P, C.POINTER(I64), C.POINTER(I64)]
    lib.sg_pool_admit.argtypes = [P, P, P, P, I64, P, P]
    lib.sg_pool_iterate.argtypes = [P, C.POINTER(I64), P]
    lib.sg_pool_finished.argtypes = [P, P, I64, C.POINTER(I64)]
    lib.sg_pool_collect.argtypes = [P, P, I64, P, P, P, P, P, P]
    for name in ("sg_pool_create", "sg_pool_info", "sg_pool_admit", "sg_pool_iterate", "sg_pool_finished",
                 "sg_pool_collect"):
        getattr(lib, name).restype = C.c_int
    lib.sg_theorem1_bound.argtypes = [I32, I32, C.POINTER(D)]
    lib.sg_theorem1_bound.restype = C.c_int
    for name in ("sg_build_grid", "sg_grid_info", "sg_solve_bvps", "sg_build_surpluses",
                 "sg_surplus_info", "sg_eval_feedback", "sg_sincos_probe"):
        getattr(lib, name).restype = C.c_int
    return lib


LIB = _load()


def _check(rc: int):
    if rc != SG_OK:
        raise SGError(f"libsg error {rc}: {LIB.sg_last_error().decode()}")


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor):
    return C.c_void_p(t.data_ptr())


def _keep_for(stream, *tensors):
    """The library queues work on `stream` and may return before it runs: when
    that is not the current stream, keep PyTorch's allocator from handing these
    tensors' blocks to the current stream's next allocations until then."""
    if stream is None or stream == torch.cuda.current_stream(stream.device):
        return
    for t in tensors:
        if t is not None:
            t.record_stream(stream)


def _dev(t, dtype, device="cuda"):
    if isinstance(t, torch.Tensor) and t.dtype == dtype and t.is_cuda and t.is_contiguous():
        # already in place: no conversion (a few microseconds per call saved)
        if (t.device.index == torch.cuda.current_device()) if device == "cuda" else (t.device == device):
            return t
    t = torch.as_tensor(t, dtype=dtype, device=device)
    return t.contiguous()


def _node_inputs(x0, T, N):
    """x0 as (n, 6) FP64, T and N as n-vectors (a scalar is broadcast), all
    contiguous on x0's device; tensors already in that form pass through."""
    x0 = _dev(x0, torch.float64)
    if x0.dim() != 2 or x0.shape[1] != 6:
        x0 = x0.reshape(-1, 6)
    n = x0.shape[0]
    T = _dev(T, torch.float64, x0.device)
    if T.dim() != 1 or T.shape[0] != n:
        T = T.reshape(-1).expand(n).contiguous()
    N = _dev(N, torch.int32, x0.device)
    if N.dim() != 1 or N.shape[0] != n:
        N = N.reshape(-1).expand(n).contiguous()
    return x0, T, N


class _DevView:
    """__cuda_array_interface__ wrapper for a borrowed device pointer."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"data": (ptr, False), "shape": tuple(shape),
                                         "typestr": typestr, "version": 3, "strides": None}


# --------------------------------------------------------------- problems
def problem_from(params, target: torch.Tensor | None = None) -> Problem:
    """Builds the ABI struct from synthetic parameters (AttitudeParams /
    LQParams / Example3Params).  target: per-node target attitudes (n, 3) on the
    device for the attitude family (kept alive by the caller while in use)."""
    p = Problem()
    if params.kind == PROBLEM_EXAMPLE3:
        p.kind = PROBLEM_EXAMPLE3
    elif params.kind == PROBLEM_ATTITUDE:
        p.kind = PROBLEM_ATTITUDE
        p.J[:] = [float(v) for v in np.asarray(params.J).ravel()]
        p.hmom[:] = [float(v) for v in np.asarray(params.hmom).ravel()]
        B = np.asarray(params.B, dtype=np.float64).reshape(3, -1)
        p.m = B.shape[1]
        B3 = np.zeros((3, 3))
        B3[:, :p.m] = B
        p.B[:] = [float(v) for v in B3.ravel()]
        if target is not None:
            if target.dtype != torch.float64 or not target.is_cuda or not target.is_contiguous():
                raise ValueError("target must be a contiguous float64 CUDA tensor (n, 3)")
            p.d_target = target.data_ptr()
        p.wv, p.ww, p.r, p.tv, p.tw = params.wv, params.ww, params.r, params.tv, params.tw
    else:
        p.kind = PROBLEM_LQ
        p.A[:] = [float(v) for v in np.asarray(params.A).ravel()]
        p.Blq[:] = [float(v) for v in np.asarray(params.B).ravel()]
        p.Q[:] = [float(v) for v in np.asarray(params.Q).ravel()]
        p.R[:] = [float(v) for v in np.asarray(params.R).ravel()]
        p.QT[:] = [float(v) for v in np.asarray(params.QT).ravel()]
    return p


# --------------------------------------------------------------- Step I
class Grid:
    """sg_build_grid handle: CGL sparse grid of dimension d and level L on a box."""

    def __init__(self, d: int, level: int, lo, hi):
        lo = np.ascontiguousarray(lo, dtype=np.float64)
        hi = np.ascontiguousarray(hi, dtype=np.float64)
        h = C.c_void_p()
        _check(LIB.sg_build_grid(d, level, lo.ctypes.data_as(C.c_void_p),
                                 hi.ctypes.data_as(C.c_void_p), C.byref(h)))
        self._h = h
        n = C.c_int64()
        dd, ll = C.c_int(), C.c_int()
        pc, pl, pi = C.c_void_p(), C.c_void_p(), C.c_void_p()
        _check(LIB.sg_grid_info(h, C.byref(n), C.byref(dd), C.byref(ll),
                                C.byref(pc), C.byref(pl), C.byref(pi)))
        self.M, self.d, self.level = n.value, dd.value, ll.value
        self.lo, self.hi = lo.copy(), hi.copy()
        self._dev = torch.device("cuda", torch.cuda.current_device())
        self._pl, self._pi = pl.value, pi.value
        self.coords = torch.as_tensor(_DevView(pc.value, (self.M, self.d), "<f8"), device=self._dev)

    @property
    def levels(self) -> torch.Tensor:
        """Borrowed (M, d) int8 view of the nodes' levels i_k."""
        return torch.as_tensor(_DevView(self._pl, (self.M, self.d), "|i1"), device=self._dev)

    @property
    def index(self) -> torch.Tensor:
        """Borrowed (M, d) int16 view of each coordinate's index in X^{i_k}."""
        return torch.as_tensor(_DevView(self._pi, (self.M, self.d), "<i2"), device=self._dev)

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) is not None and LIB is not None:
            LIB.sg_grid_free(self._h)
            self._h = None


# --------------------------------------------------------------- Step II
def workspace_bytes(n: int, n_max: int, precision: int = PREC_FP64) -> int:
    return int(LIB.sg_solve_workspace_bytes(n, n_max, precision))


def solve_bvps(problem: Problem, x0: torch.Tensor, T, N, *, tol=1e-8, max_iter=50,
               precision=PREC_FP64, damping=True, n_max=None, return_Y=False,
               workspace: torch.Tensor | None = None, persistent=False, blocks_per_sm=0,
               graph=False, out=None, Y0: torch.Tensor | None = None, cond_warps=4, stream=None):
    """sg_solve_bvps on device tensors.  x0 (n, 6) f64; T (n,) f64; N (n,) int32.
    `out` may hold preallocated output tensors (keys lambda0, u0, V, status,
    iters); reusing them (and the workspace) lets graph=True replay one graph.
    graph: 0 host loop, 1 (or True) one cached graph, 2 one graph per mesh size.
    Y0 (n, 3 n_max + 1, 12) f64: warm start from this iterate; it is
    overwritten with the final iterate (and returned as "Y").
    With graph != 0 the call returns once the work is queued on `stream`
    (default: the current stream): read the outputs in that stream's order."""
    x0, T, N = _node_inputs(x0, T, N)
    n = x0.shape[0]
    dev = x0.device
    if n_max is None:
        n_max = int(N.max().item()) if n else 1
    if workspace is None:
        workspace = torch.empty(max(workspace_bytes(n, n_max, precision), 1), dtype=torch.uint8,
                                device=dev)
    if out is None:
        out = {
            "lambda0": torch.empty((n, 6), dtype=torch.float64, device=dev),
            "u0": torch.empty((n, 3), dtype=torch.float64, device=dev),
            "V": torch.empty((n,), dtype=torch.float64, device=dev),
            "status": torch.empty((n,), dtype=torch.int32, device=dev),
            "iters": torch.empty((n,), dtype=torch.int32, device=dev),
        }
    if Y0 is not None:
        if tuple(Y0.shape) != (n, 3 * n_max + 1, 12) or Y0.dtype != torch.float64 or not Y0.is_contiguous():
            raise ValueError("Y0 must be a contiguous (n, 3 n_max + 1, 12) float64 tensor")
        Y = Y0
    else:
        Y = torch.zeros((n, 3 * n_max + 1, 12), dtype=torch.float64, device=dev) if return_Y else None
    opts = SolveOpts(tol=tol, max_iter=max_iter, precision=precision, damping=int(bool(damping)),
                     persistent=int(bool(persistent)), blocks_per_sm=int(blocks_per_sm),
                     graph=int(graph), warm_start=int(Y0 is not None), cond_warps=int(cond_warps))
    _check(LIB.sg_solve_bvps(C.byref(problem), _ptr(x0), n, _ptr(T), _ptr(N), n_max, C.byref(opts),
                             _ptr(workspace), workspace.numel(), _ptr(out["lambda0"]), _ptr(out["u0"]),
                             _ptr(out["V"]), _ptr(out["status"]), _ptr(out["iters"]),
                             _ptr(Y) if Y is not None else None, _stream(stream)))
    _keep_for(stream, x0, T, N, workspace, Y, *out.values())
    if Y is not None:
        out["Y"] = Y
    return out


FORM_NAMES = ["phase-host-loop", "phase-graph", "phase-graph-per-mesh", "phase-graph-per-mesh-cond2",
              "phase-graph-per-mesh-cond8", "persistent-graph", "persistent-graph-1blk"]


def autotune_solve(problem: Problem, x0, T, N, *, tol=1e-8, max_iter=50, precision=PREC_FP64,
                   damping=True, n_max=None, workspace=None, force=False, stream=None):
    """sg_autotune_solve: returns (best options as a dict, {form name: ms})."""
    x0, T, N = _node_inputs(x0, T, N)
    n = x0.shape[0]
    dev = x0.device
    if n_max is None:
        n_max = int(N.max().item()) if n else 1
    if workspace is None:
        workspace = torch.empty(max(workspace_bytes(n, n_max, precision), 1), dtype=torch.uint8, device=dev)
    outs = [torch.empty((n, 6), dtype=torch.float64, device=dev), torch.empty((n, 3), dtype=torch.float64, device=dev),
            torch.empty((n,), dtype=torch.float64, device=dev), torch.empty((n,), dtype=torch.int32, device=dev),
            torch.empty((n,), dtype=torch.int32, device=dev)]
    base = SolveOpts(tol=tol, max_iter=max_iter, precision=precision, damping=int(bool(damping)))
    best = SolveOpts()
    nc = len(FORM_NAMES)
    ms = (C.c_double * nc)(*([float("nan")] * nc))
    _check(LIB.sg_autotune_solve(C.byref(problem), _ptr(x0), n, _ptr(T), _ptr(N), n_max, C.byref(base),
                                 _ptr(workspace), workspace.numel(), *[_ptr(t) for t in outs], C.byref(best),
                                 ms, int(bool(force)), _stream(stream)))
    choice = {"persistent": bool(best.persistent), "graph": int(best.graph), "blocks_per_sm": best.blocks_per_sm,
              "cond_warps": int(best.cond_warps)}
    return choice, {FORM_NAMES[i]: ms[i] for i in range(nc)}


class SolverPool:
    """sg_pool_*: resident Newton state for `slots` nodes; solves join and
    leave between iterations (continuous batching).  The workspace is a torch
    allocation owned by this object."""

    def __init__(self, problem: Problem, slots: int, n_max: int, *, tol=1e-8, max_iter=50,
                 precision=PREC_MIXED, damping=True, device=None, stream=None):
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.slots, self.n_max, self.precision = int(slots), int(n_max), precision
        nbytes = int(LIB.sg_pool_workspace_bytes(self.slots, self.n_max, precision))
        if nbytes == 0:
            raise SGError("sg_pool_workspace_bytes: invalid pool size or precision")
        self.nbytes = nbytes
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self._problem = problem   # kept alive with the handle
        opts = SolveOpts(tol=tol, max_iter=max_iter, precision=precision, damping=int(bool(damping)))
        h = C.c_void_p()
        _check(LIB.sg_pool_create(C.byref(problem), self.slots, self.n_max, C.byref(opts), _ptr(self.workspace),
                                  nbytes, C.byref(h), _stream(stream)))
        self._h = h

    def info(self):
        f, b = C.c_int64(), C.c_int64()
        _check(LIB.sg_pool_info(self._h, C.byref(f), C.byref(b)))
        return f.value, b.value

    def admit(self, x0, T, N, stream=None) -> np.ndarray:
        """Admits the solves of the rows of x0; returns their slots (int64).
        Raises SGError with code SG_EFULL when too few slots are free."""
        x0 = _dev(x0, torch.float64, self.device).reshape(-1, 6)
        n = x0.shape[0]
        T = _dev(T, torch.float64, self.device).reshape(-1).expand(n).contiguous()
        N = _dev(N, torch.int32, self.device).reshape(-1).expand(n).contiguous()
        slots = np.empty(n, dtype=np.int64)
        rc = LIB.sg_pool_admit(self._h, _ptr(x0), _ptr(T), _ptr(N), n, slots.ctypes.data_as(C.c_void_p),
                               _stream(stream))
        if rc == SG_EFULL:
            raise SGError(f"libsg error {rc}: {LIB.sg_last_error().decode()}")
        _check(rc)
        return slots

    def iterate(self, stream=None) -> int:
        """One Newton iteration of every slot in progress; returns how many still iterate."""
        a = C.c_int64()
        _check(LIB.sg_pool_iterate(self._h, C.byref(a), _stream(stream)))
        return a.value

    def finished(self) -> np.ndarray:
        out = np.empty(self.slots, dtype=np.int64)
        c = C.c_int64()
        _check(LIB.sg_pool_finished(self._h, out.ctypes.data_as(C.c_void_p), self.slots, C.byref(c)))
        return out[:c.value].copy()

    def collect(self, slots, out=None, stream=None) -> dict:
        """Outputs of the finished `slots` (row j = slots[j]); frees them."""
        slots = np.ascontiguousarray(slots, dtype=np.int64)
        n = slots.shape[0]
        if out is None:
            out = {"lambda0": torch.empty((n, 6), dtype=torch.float64, device=self.device),
                   "u0": torch.empty((n, 3), dtype=torch.float64, device=self.device),
                   "V": torch.empty((n,), dtype=torch.float64, device=self.device),
                   "status": torch.empty((n,), dtype=torch.int32, device=self.device),
                   "iters": torch.empty((n,), dtype=torch.int32, device=self.device)}
        _check(LIB.sg_pool_collect(self._h, slots.ctypes.data_as(C.c_void_p), n, _ptr(out["lambda0"]),
                                   _ptr(out["u0"]), _ptr(out["V"]), _ptr(out["status"]), _ptr(out["iters"]),
                                   _stream(stream)))
        return out

    def __del__(self):
        if getattr(self, "_h", None) is not None and LIB is not None:
            LIB.sg_pool_free(self._h)
            self._h = None


# --------------------------------------------------------------- Step III
class Surplus:
    """sg_build_surpluses handle: hierarchical surpluses of values at the nodes.
    The build is queued on `stream` (default: the current stream); use the
    handle on another stream only after an event or a synchronisation."""

    def __init__(self, grid: Grid, values: torch.Tensor, stream=None):
        values = _dev(values, torch.float64).reshape(grid.M, -1)
        h = C.c_void_p()
        _check(LIB.sg_build_surpluses(grid.handle, _ptr(values), values.shape[1], C.byref(h),
                                      _stream(stream)))
        _keep_for(stream, values)
        self._h = h
        n, k, pw = C.c_int64(), C.c_int(), C.c_void_p()
        _check(LIB.sg_surplus_info(h, C.byref(n), C.byref(k), C.byref(pw)))
        self.M, self.k = n.value, k.value
        self.d = grid.d
        dev = torch.device("cuda", torch.cuda.current_device())
        self.W = torch.as_tensor(_DevView(pw.value, (self.M, self.k), "<f8"), device=dev)

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) is not None and LIB is not None:
            LIB.sg_surplus_free(self._h)
            self._h = None


def eval_feedback(surplus: Surplus, xq: torch.Tensor, mode: int = EVAL_FP64,
                  out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    xq = _dev(xq, torch.float64).reshape(-1, surplus.d)
    Q = xq.shape[0]
    if out is None:
        out = torch.empty((Q, surplus.k), dtype=torch.float64, device=xq.device)
    _check(LIB.sg_eval_feedback(surplus.handle, _ptr(xq), Q, mode, _ptr(out), _stream(stream)))
    _keep_for(stream, xq, out)
    return out


def theorem1_bound(d: int, q: int) -> float:
    """sg_theorem1_bound: the Theorem 1 factor bounding |e_bvp| / eps."""
    out = C.c_double()
    _check(LIB.sg_theorem1_bound(d, q, C.byref(out)))
    return out.value


def mc_error_amplification(d: int, level: int, n_points: int, seed: int = 0, symmetric: bool = False,
                           mode: int = EVAL_DF32, device="cuda") -> float:
    """Monte-Carlo estimate of |e_bvp| / eps (Section 4.2, Eq. ebvp_explicit2):
    the interpolant of independent nodal errors drawn uniformly from [0, 1]
    (as printed; [-1, 1] with symmetric=True), maximised over n_points uniform
    points of [0, 1]^d.  Grid, surpluses and evaluation run in the library."""
    lo, hi = np.zeros(d), np.ones(d)
    g = Grid(d, level, lo, hi)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    eps = torch.rand((g.M, 1), generator=gen, dtype=torch.float64)
    if symmetric:
        eps = 2.0 * eps - 1.0
    xq = torch.rand((n_points, d), generator=gen, dtype=torch.float64)
    S = Surplus(g, eps.to(device))
    e = eval_feedback(S, xq.to(device), mode=mode)
    return float(e.abs().max().item())


def attitude_targets(problem: Problem, x0: torch.Tensor, stream=None):
    """sg_attitude_targets: Example II target attitudes (n, 3) and status (n,)."""
    x0 = _dev(x0, torch.float64).reshape(-1, 6)
    n = x0.shape[0]
    tgt = torch.empty((n, 3), dtype=torch.float64, device=x0.device)
    st = torch.empty((n,), dtype=torch.int32, device=x0.device)
    _check(LIB.sg_attitude_targets(C.byref(problem), _ptr(x0), n, _ptr(tgt), _ptr(st), _stream(stream)))
    return tgt, st


def sincos_probe(x: torch.Tensor, stream=None):
    """sg_sincos_probe: the library's FP64 sine and cosine at x (device)."""
    x = _dev(x, torch.float64).reshape(-1)
    s, c = torch.empty_like(x), torch.empty_like(x)
    _check(LIB.sg_sincos_probe(_ptr(x), x.numel(), _ptr(s), _ptr(c), _stream(stream)))
    return s, c


# --------------------------------------------------------------- closed loop
def simulate_closed_loop(problem: Problem, surplus: Surplus, x0, nsteps: int, dt: float,
                         mode: int = EVAL_DF32, keep_trajectory=False, stream=None):
    """sg_simulate_closed_loop: returns dict with xT (n, 6), cost (n,) and,
    if asked, traj (n, nsteps+1, 6) and ctrl (n, nsteps, 3)."""
    x0 = _dev(x0, torch.float64).reshape(-1, 6)
    n = x0.shape[0]
    dev = x0.device
    out = {"xT": torch.empty((n, 6), dtype=torch.float64, device=dev),
           "cost": torch.empty((n,), dtype=torch.float64, device=dev)}
    if keep_trajectory:
        out["traj"] = torch.empty((n, nsteps + 1, 6), dtype=torch.float64, device=dev)
        out["ctrl"] = torch.empty((n, nsteps, 3), dtype=torch.float64, device=dev)
    _check(LIB.sg_simulate_closed_loop(C.byref(problem), surplus.handle, _ptr(x0), n, nsteps, dt, mode,
                                       _ptr(out["xT"]), _ptr(out["cost"]),
                                       _ptr(out["traj"]) if keep_trajectory else None,
                                       _ptr(out["ctrl"]) if keep_trajectory else None, _stream(stream)))
    return out

