"""Pins of the oracle's closed-loop simulation (zero-order hold + RK4)."""
import numpy as np
from scipy.linalg import expm, solve_continuous_are

import synth
from oracle import closed_loop as cl
from oracle import grid as G
from oracle import interp as I
from oracle import problems as P


def _lq_linear_feedback():
    params = synth.lq_params(0)
    pr = P.make(params)
    g = G.Grid(6, 1, *synth.box())
    # the infinite-horizon LQ gain: a stabilising linear feedback
    P_inf = solve_continuous_are(pr.A, pr.B, pr.Q, pr.R)
    K = np.linalg.solve(pr.R, pr.B.T @ P_inf)
    # the feedback u = -K x is linear, so the level-1 interpolant reproduces it exactly
    w = I.surpluses(g, -(g.x @ K.T))
    return pr, g, w, K


def test_interpolant_reproduces_linear_feedback():
    pr, g, w, K = _lq_linear_feedback()
    xq = synth.uniform_queries(20, g.lo, g.hi, seed=4)
    assert np.allclose(I.eval_surplus(g, w, xq), -(xq @ K.T), atol=1e-13)


def test_zero_order_hold_matches_exact_discretisation():
    """Over one hold interval with u constant the plant is linear, and the exact
    step is x+ = Phi x + Gamma u with [[Phi, Gamma], [0, I]] = expm([[A, B], [0, 0]] dt);
    RK4 reproduces it to O(dt^5) per step."""
    pr, g, w, K = _lq_linear_feedback()
    x0 = np.array([0.3, -0.2, 0.1, 0.25, -0.15, 0.05])
    errs = []
    for dt, n in ((0.01, 300), (0.005, 600)):
        xs, us, _ = cl.simulate(pr, g, w, x0, n, dt)
        Mblk = np.zeros((9, 9))
        Mblk[:6, :6] = pr.A
        Mblk[:6, 6:] = pr.B
        E = expm(Mblk * dt)
        Phi, Gam = E[:6, :6], E[:6, 6:]
        x = x0.copy()
        for _ in range(n):
            x = Phi @ x + Gam @ (-K @ x)
        errs.append(np.max(np.abs(xs[-1] - x)))
    assert errs[0] <= 1e-9 * np.max(np.abs(x0))
    assert errs[0] / errs[1] > 12      # fourth order in dt


def test_rk4_fourth_order_under_step_halving():
    """Attitude plant with a constant held control: the RK4 error shrinks by
    about 2^4 per halving of dt (reference: a much finer RK4)."""
    pr = P.make(synth.attitude_params(0))
    u = np.array([0.2, -0.1, 0.05])
    x0 = np.array([0.3, -0.2, 0.4, 0.1, -0.3, 0.2])

    def run(dt, T=1.0):
        x = x0.copy()
        for _ in range(int(round(T / dt))):
            k1 = cl.plant_rhs(pr, x, u)
            k2 = cl.plant_rhs(pr, x + 0.5 * dt * k1, u)
            k3 = cl.plant_rhs(pr, x + 0.5 * dt * k2, u)
            k4 = cl.plant_rhs(pr, x + dt * k3, u)
            x = x + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        return x

    ref = run(1e-3)
    e1 = np.max(np.abs(run(0.1) - ref))
    e2 = np.max(np.abs(run(0.05) - ref))
    assert 12 < e1 / e2 < 20


def test_closed_loop_cost_is_quadrature_of_running_cost():
    """z(T) from the RK4 stages equals the trapezoid-free quadrature of L along a
    trajectory whose state and control are known exactly: the origin stays put
    with zero control and zero cost."""
    pr, g, w, K = _lq_linear_feedback()
    xs, us, z = cl.simulate(pr, g, w, np.zeros(6), 50, 0.01)
    assert z == 0.0 and np.all(xs == 0.0)
