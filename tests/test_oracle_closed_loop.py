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


# ------------------------------------------------------------------ attitude branch
def _lambda_for(pr, u, rng):
    """A costate whose minimiser of H is u: u*(x, lambda) = -B' J^-1 lambda_w / r,
    so lambda_w = -r J B'^-1 u (B invertible); lambda_v is free."""
    lw = -pr.p.r * np.asarray(pr.p.J) * np.linalg.solve(pr.B.T, u)
    return np.concatenate([rng.standard_normal(3), lw])


def _attitude_pin(plant_rhs, running_cost_xu, seed=0, target=None):
    """The largest deviation of plant_rhs and running_cost_xu from the pinned
    Hamiltonian of problems.Attitude, at random (x, u):
      f(x, u) = dH*/dlambda at the lambda whose minimiser is u (envelope
      theorem: u* makes dH/du vanish), by complex-step differentiation;
      L(x, u) = running_cost at that (x, lambda)."""
    pr = P.make(synth.attitude_params(0), target=target)
    rng = np.random.default_rng(seed)
    dev = 0.0
    for _ in range(8):
        x = rng.uniform(-0.7, 0.7, 6)
        u = rng.standard_normal(3)
        lam = _lambda_for(pr, u, rng)
        y = np.concatenate([x, lam])
        assert np.allclose(pr.ustar(x, lam), u, atol=1e-13)
        dH = np.empty(6)
        for c in range(6):
            yc = y.astype(np.complex128)
            yc[6 + c] += 1e-30j
            dH[c] = pr.hamiltonian(yc).imag / 1e-30
        f = plant_rhs(pr, x, u)
        dev = max(dev, np.max(np.abs(f - dH)) / max(1.0, np.max(np.abs(dH))))
        L = running_cost_xu(pr, x, u)
        Lref = pr.running_cost(y)
        dev = max(dev, abs(L - Lref) / max(1.0, abs(Lref)))
    return dev


def test_attitude_plant_and_cost_match_the_hamiltonian():
    assert _attitude_pin(cl.plant_rhs, cl.running_cost_xu) <= 1e-13
    # with a target attitude (Example II's running cost penalises v - v_e)
    assert _attitude_pin(cl.plant_rhs, cl.running_cost_xu, seed=1, target=[0.1, -0.2, 0.05]) <= 1e-13


def test_planted_closed_loop_mistakes_are_caught():
    """A sign error in the control term of the plant, a dropped 1/J on it, and
    the control weight left out of the cost each fail the pin."""
    def plant_sign(pr, x, u):
        f = pr.f0(x[:, None])[:, 0]
        f[3:] = f[3:] - pr.Jinv * (pr.B @ u)
        return f

    def plant_noJ(pr, x, u):
        f = pr.f0(x[:, None])[:, 0]
        f[3:] = f[3:] + pr.B @ u
        return f

    def cost_no_r(pr, x, u):
        return 0.5 * (pr.p.wv * x[:3] @ x[:3] + pr.p.ww * x[3:6] @ x[3:6] + u @ u)

    assert _attitude_pin(plant_sign, cl.running_cost_xu) > 1e-3
    assert _attitude_pin(plant_noJ, cl.running_cost_xu) > 1e-3
    assert _attitude_pin(cl.plant_rhs, cost_no_r) > 1e-3
