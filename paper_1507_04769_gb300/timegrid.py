"""Time as a grid dimension (Section 5, Example III).

The characteristic BVP of a time-invariant problem started at (t0, x0) on
[t0, T] is the same problem started at x0 over the horizon T - t0, so the
value function V(t, x) and the feedback u*(t, x) come from one batched solve
over a sparse grid in (t, x) space: node (t, x) is solved from x over the
horizon T - t.  The surpluses of V and u* over that grid give the
interpolant in (t, x) that a variable-horizon MPC feeds back.

Every step runs in the library: the grid (sg_build_grid), the solves
(sg_solve_bvps), the surpluses (sg_build_surpluses) and the evaluation
(sg_eval_feedback).  This module only marshals the (t, x) layout.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import sg, surfaces


@dataclass
class ValueSurface:
    grid: sg.Grid              # d = 1 + n_state, coordinates (t, x)
    surplus: sg.Surplus        # k = 2 outputs: V and u*_1
    result: dict               # per-node solve outputs (lambda0, u0, V, status, iters)
    continued: int             # nodes re-solved by continuation in the horizon
    t_end: float
    horizons: np.ndarray       # t_end - t per node
    intervals: np.ndarray      # mesh intervals per node

    def evaluate(self, tx, mode: int = sg.EVAL_DF32) -> torch.Tensor:
        """(V, u*) at query points tx (Q x d, columns (t, x))."""
        return sg.eval_feedback(self.surplus, tx, mode=mode)


def solve_value_surface(problem: sg.Problem, n_state: int, level: int, lo, hi, t_end: float, mesh,
                        precision: int = sg.PREC_MIXED, tol: float = 1e-8, max_iter: int = 100,
                        continuation=((0.25, 0.5, 0.75, 1.0), tuple(k / 10 for k in range(1, 11))),
                        device="cuda") -> ValueSurface:
    """Solves the characteristic BVP at every node of the level-`level` CGL
    sparse grid on the (t, x) box [lo, hi] (lo[0], hi[0]: the time range,
    hi[0] <= t_end) and builds the surpluses of V and u*_1.  Raises if a node
    does not converge (its value would spoil the whole interpolant).

    mesh(horizons) -> intervals per node (numpy int32).

    Nodes whose damped Newton iteration stalls from the zero-control guess
    (Example III has about 1 % of them at long horizons: the Armijo search
    settles on a non-root minimum of |F|^2) are re-solved by continuation in
    the horizon: the same mesh over the horizons `continuation` x (t_end - t)
    in turn, each solve warm-started from the previous one's collocation
    solution (the mesh points map onto each other, only h changes); nodes
    that still stall take the next, finer schedule."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    d = lo.size
    if d != 1 + n_state or not 1 <= n_state <= 6:
        raise ValueError("the box must be (t, x) with 1 <= n_state <= 6")
    if hi[0] > t_end:
        raise ValueError("the time range must end at or before t_end")
    g = sg.Grid(d, level, lo, hi)
    coords = g.coords
    M = g.M
    x0 = torch.zeros((M, 6), dtype=torch.float64, device=device)
    x0[:, :n_state] = coords[:, 1:]
    tau_d = (t_end - coords[:, 0]).clamp_min(0.0).contiguous()
    tau = tau_d.cpu().numpy()
    N = np.asarray(mesh(tau), dtype=np.int32)
    N_d = torch.as_tensor(N, device=device)
    res, n_continued = surfaces.solve_nodes(problem, x0, tau_d, N_d, precision=precision, tol=tol,
                                            max_iter=max_iter, schedules=continuation)
    bad = int((res["status"] != sg.CONVERGED).sum().item())
    if bad:
        raise RuntimeError(f"{bad} of {M} nodes did not converge (max_iter = {max_iter}, with continuation)")
    vals = torch.stack([res["V"], res["u0"][:, 0]], dim=1).contiguous()
    S = sg.Surplus(g, vals)
    return ValueSurface(grid=g, surplus=S, result=res, continued=n_continued, t_end=t_end,
                        horizons=tau, intervals=N)
