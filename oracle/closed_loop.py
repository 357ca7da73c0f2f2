"""Oracle: closed-loop simulation with the interpolated feedback.

TEST INFRASTRUCTURE ONLY (see oracle/grid.py).

The on-line phase of Section 3.3 feeds u*(x), interpolated from the sparse
grid, back into the plant.  Section 5 simulates model predictive control with
a zero-order hold: the control is computed from the measured state at each
sampling instant and held until the next one.  Here: at t_k = k dt,
u_k = I^q(u*)(x_k); over [t_k, t_k + dt] the plant x' = f(x, u_k) is advanced
by one classical fourth-order Runge-Kutta step, together with the running
cost z' = L(x, u_k), z(0) = 0.
"""
from __future__ import annotations

import numpy as np

from . import interp


def plant_rhs(prob, x, u):
    """f(x, u) for a fixed control u (control-affine plants of problems.py)."""
    if hasattr(prob, "Jinv"):
        f = prob.f0(x[:, None])[:, 0]
        f[3:] = f[3:] + prob.Jinv * (prob.B @ u)
        return f
    return prob.A @ x + prob.B @ u


def running_cost_xu(prob, x, u):
    """L(x, u) for a given control u (the running cost of problems.py, whose
    running_cost takes u = u*(x, lambda))."""
    if hasattr(prob, "Jinv"):
        p = prob.p
        dv = x[:3] - prob.target
        return 0.5 * (p.wv * dv @ dv + p.ww * x[3:6] @ x[3:6] + p.r * u @ u)
    return 0.5 * (x @ prob.Q @ x + u @ prob.R @ u)


def simulate(prob, grid, w, x0, nsteps, dt):
    """One trajectory: returns (states (nsteps+1, 6), controls (nsteps, m), cost)."""
    x = np.asarray(x0, dtype=np.float64).copy()
    xs = [x.copy()]
    us = []
    z = 0.0
    for _ in range(nsteps):
        u = interp.eval_surplus(grid, w, x[None, :])[0]
        k1 = plant_rhs(prob, x, u)
        l1 = running_cost_xu(prob, x, u)
        x2 = x + 0.5 * dt * k1
        k2 = plant_rhs(prob, x2, u)
        l2 = running_cost_xu(prob, x2, u)
        x3 = x + 0.5 * dt * k2
        k3 = plant_rhs(prob, x3, u)
        l3 = running_cost_xu(prob, x3, u)
        x4 = x + dt * k3
        k4 = plant_rhs(prob, x4, u)
        l4 = running_cost_xu(prob, x4, u)
        x = x + (dt / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
        z = z + (dt / 6.0) * (l1 + 2 * l2 + 2 * l3 + l4)
        xs.append(x.copy())
        us.append(u)
    return np.array(xs), np.array(us), z
