"""Batched node solves with continuation, and the value surface of the
two-wheel attitude problem (Section 5, Example II).

`solve_nodes` runs sg_solve_bvps over a set of initial states in batches
that bound the workspace, and re-solves the nodes whose damped Newton
iteration stalls from the zero-control guess by continuation in the horizon:
the same mesh over fractions of the horizon in turn, each solve warm-started
from the previous collocation solution (only h changes, the mesh points map
onto each other).  Per-node target attitudes (Example II) travel with the
batch.  Every step runs in the library; this module only keeps the
bookkeeping.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import sg

SCHEDULES = ((0.25, 0.5, 0.75, 1.0), tuple(k / 10 for k in range(1, 11)))


def _with_target(problem: sg.Problem, target: torch.Tensor | None) -> sg.Problem:
    p = type(problem).from_buffer_copy(problem)
    p.d_target = target.data_ptr() if target is not None else None
    return p


def solve_nodes(problem: sg.Problem, x0: torch.Tensor, T: torch.Tensor, N: torch.Tensor, *,
                target: torch.Tensor | None = None, precision: int = sg.PREC_MIXED, tol: float = 1e-8,
                max_iter: int = 100, schedules=SCHEDULES, batch_nodes: int = 1 << 14):
    """Solves every node; returns (outputs dict, number of nodes continued).
    x0 (n, 6), T (n,), N (n,) int32, target (n, 3) or None, all on the device."""
    n = x0.shape[0]
    dev = x0.device
    out = {"lambda0": torch.empty((n, 6), dtype=torch.float64, device=dev),
           "u0": torch.empty((n, 3), dtype=torch.float64, device=dev),
           "V": torch.empty((n,), dtype=torch.float64, device=dev),
           "status": torch.empty((n,), dtype=torch.int32, device=dev),
           "iters": torch.empty((n,), dtype=torch.int32, device=dev)}

    def run(idx, scale=1.0, Y=None, keep_y=False):
        tg = target[idx].contiguous() if target is not None else None
        Ns = N[idx].contiguous()
        return sg.solve_bvps(_with_target(problem, tg), x0[idx].contiguous(), (T[idx] * scale).contiguous(), Ns,
                             tol=tol, max_iter=max_iter, precision=precision, n_max=int(Ns.max().item()),
                             Y0=Y, return_Y=keep_y)

    for b0 in range(0, n, batch_nodes):
        idx = torch.arange(b0, min(n, b0 + batch_nodes), device=dev)
        r = run(idx)
        for k in out:
            out[k][idx] = r[k]
    continued = int((out["status"] != sg.CONVERGED).sum().item())
    for schedule in schedules:   # finer schedules for the nodes that still stall
        idx = torch.nonzero(out["status"] != sg.CONVERGED).flatten()
        if not idx.numel():
            break
        for b0 in range(0, idx.numel(), batch_nodes):
            sub = idx[b0:b0 + batch_nodes]
            Y = None
            for scale in schedule:
                r = run(sub, scale, Y, keep_y=True)
                Y = r["Y"]
            for k in out:
                out[k][sub] = r[k]
    return out, continued


@dataclass
class AttitudeSurface:
    grid: sg.Grid
    surplus: sg.Surplus        # k = 3 outputs: u*_1, u*_2, V
    targets: torch.Tensor      # (M, 3) target attitude per node
    result: dict
    continued: int
    T: float

    def evaluate(self, x, mode: int = sg.EVAL_DF32) -> torch.Tensor:
        return sg.eval_feedback(self.surplus, x, mode=mode)


def two_wheel_surface(params, level: int, lo, hi, T: float, h: float = 5.0 / 32.0,
                      precision: int = sg.PREC_MIXED, tol: float = 1e-8, batch_nodes: int = 1 << 14,
                      device="cuda") -> AttitudeSurface:
    """Example II: the CGL sparse grid of the given level on the box [lo, hi] of
    (v, w), the target attitude of every node (sg_attitude_targets), the
    characteristic BVP over [0, T] with N = T / h intervals, and the surpluses
    of (u*_1, u*_2, V).  Raises if a node has no target or does not converge."""
    g = sg.Grid(6, level, np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64))
    x0 = g.coords.contiguous()
    base = sg.problem_from(params)
    tgt, st = sg.attitude_targets(base, x0)
    if int((st != 0).sum().item()):
        raise RuntimeError(f"{int((st != 0).sum().item())} nodes have no target attitude")
    Nn = max(1, int(round(T / h)))
    Td = torch.full((g.M,), float(T), dtype=torch.float64, device=device)
    Nd = torch.full((g.M,), Nn, dtype=torch.int32, device=device)
    res, continued = solve_nodes(base, x0, Td, Nd, target=tgt, precision=precision, tol=tol,
                                 batch_nodes=batch_nodes)
    bad = int((res["status"] != sg.CONVERGED).sum().item())
    if bad:
        raise RuntimeError(f"{bad} of {g.M} nodes did not converge")
    vals = torch.stack([res["u0"][:, 0], res["u0"][:, 1], res["V"]], dim=1).contiguous()
    return AttitudeSurface(grid=g, surplus=sg.Surplus(g, vals), targets=tgt, result=res, continued=continued, T=T)
