"""Oracle pins for Example II (Section 5): the optimal trajectory printed in
the paper's figure from x(0) = (0, pi/8, 0, 0, 0, 0), the target attitude of
Eq. optim_attitude, and the invariant of the reachable manifold.  The
printed trajectory pins the attitude conventions (E, R, S), the two-wheel
control and the costs together."""
import os

import numpy as np
import pytest

import synth
from oracle import bvp, lobatto
from oracle import problems as P

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "example2_trajectory.txt")
PRM = synth.example2_params()
X0 = np.array([0.0, np.pi / 8, 0.0, 0.0, 0.0, 0.0])
N = 960   # mesh width 1/32: the dense output between mesh points is O(h^4)


def _printed():
    rows = [list(map(float, l.split())) for l in open(GOLDEN) if l.strip() and l[0] != "#"]
    return np.array(rows)


def _dense(Y, T, N, t):
    """The Lobatto IIIA collocation polynomial (cubic through the four stage
    values of the interval) at time t."""
    _, _, c = lobatto.tableau()
    h = T / N
    i = min(int(t / h), N - 1)
    tau = (t - i * h) / h
    pts = Y[3 * i:3 * i + 4]
    out = np.zeros(Y.shape[1])
    for k in range(4):
        lk = np.prod([(tau - c[j]) / (c[k] - c[j]) for j in range(4) if j != k])
        out += lk * pts[k]
    return out


@pytest.fixture(scope="module")
def solution():
    ve = P.target_attitude(PRM, X0)
    pr = P.make(PRM, target=ve)
    return ve, pr, bvp.solve(pr, X0, synth.EXAMPLE2_T, N, tol=1e-12)


def test_target_attitude_satisfies_constraint_and_is_a_maximum(solution):
    ve, _, _ = solution
    B, J, H = np.asarray(PRM.B), np.asarray(PRM.J), np.asarray(PRM.hmom)
    C = P.reachable_normal(B)
    assert np.allclose(C @ B, 0.0, atol=1e-15)
    rhs = C @ (J * X0[3:] - P.rot(X0[:3]) @ H)
    assert abs(-C @ P.rot(ve) @ H - rhs) < 1e-12
    # no feasible neighbour (projected onto the constraint) has a larger trace
    rng = np.random.default_rng(1)
    g = np.array([(-C @ P.rot(ve + 1e-6 * e) @ H + C @ P.rot(ve - 1e-6 * e) @ H) / 2e-6 for e in np.eye(3)])
    for _ in range(20):
        d = rng.standard_normal(3)
        d -= g * (d @ g) / (g @ g)
        d *= 1e-3 / np.linalg.norm(d)
        assert np.trace(P.rot(ve + d)) <= np.trace(P.rot(ve)) + 1e-9


def test_printed_optimal_trajectory(solution):
    """The printed trajectory (16 times, 8 components) to 1e-6."""
    _, _, s = solution
    assert s.status == bvp.CONVERGED
    pr = _printed()
    for row in pr:
        t, ref = row[0], row[1:]
        y = _dense(s.Y, synth.EXAMPLE2_T, N, t)
        u = -np.asarray(PRM.B).T @ (y[9:12] / np.asarray(PRM.J)) / PRM.r
        got = np.concatenate([y[:6], u])
        assert np.abs(got - ref).max() < 1e-6, (t, got, ref)


def test_reachable_manifold_is_invariant(solution):
    """C'(J w - R(v) H) is conserved along any controlled trajectory (C'B = 0),
    so v_e is constant along the solution."""
    _, _, s = solution
    B, J, H = np.asarray(PRM.B), np.asarray(PRM.J), np.asarray(PRM.hmom)
    C = P.reachable_normal(B)
    q = np.array([C @ (J * y[3:6] - P.rot(y[:3]) @ H) for y in s.Y])
    assert np.abs(q - q[0]).max() < 1e-9


def test_planted_convention_error_fails_printed_trajectory():
    """S(w) a = w x a instead of a x w: the printed trajectory is not reproduced."""
    class Flipped(P.Attitude):
        def f0(self, x):
            f = super().f0(x)
            f[3:6] = -f[3:6]
            return f

        def grad_lf0(self, x, lam):
            g = super().grad_lf0(x, np.concatenate([lam[:3], np.zeros_like(lam[3:6])]))
            gw = super().grad_lf0(x, np.concatenate([np.zeros_like(lam[:3]), lam[3:6]]))
            return g - gw

    ve = P.target_attitude(PRM, X0)
    s = bvp.solve(Flipped(PRM, target=ve), X0, synth.EXAMPLE2_T, N, tol=1e-10)
    u0 = -np.asarray(PRM.B).T @ (s.Y[0, 9:12] / np.asarray(PRM.J)) / PRM.r
    assert np.abs(u0 - _printed()[0, 7:9]).max() > 1e-3


def _slsqp_target(x0, starts):
    """A generic constrained optimiser on Eq. optim_attitude (independent of the
    closed form): SLSQP from several starts, the largest trace kept."""
    from scipy.optimize import minimize
    B, J, H = np.asarray(PRM.B), np.asarray(PRM.J), np.asarray(PRM.hmom)
    C = P.reachable_normal(B)
    rhs = C @ (J * x0[3:] - P.rot(x0[:3]) @ H)
    cons = {"type": "eq", "fun": lambda v: -C @ P.rot(v) @ H - rhs}
    best = None
    for g in starts:
        r = minimize(lambda v: -np.trace(P.rot(v)), g, constraints=[cons], method="SLSQP", tol=1e-15,
                     options={"maxiter": 500})
        if r.success and abs(cons["fun"](r.x)) < 1e-10 and (best is None or r.fun < best.fun):
            best = r
    return best.x


def test_target_attitude_matches_a_generic_optimiser():
    """At random states of the Example II box the closed form and SLSQP agree:
    the same trace to 1e-12 (SLSQP never finds a larger one) and the same angles
    to the optimiser's accuracy on the flat maximum (1e-6)."""
    lo, hi = synth.example2_box()
    rng = np.random.default_rng(3)
    for _ in range(6):
        x0 = rng.uniform(lo, hi)
        ve = P.target_attitude(PRM, x0)
        vs = _slsqp_target(x0, (x0[:3], np.zeros(3), ve + 0.1))
        assert np.trace(P.rot(vs)) <= np.trace(P.rot(ve)) + 1e-12
        assert abs(np.trace(P.rot(vs)) - np.trace(P.rot(ve))) < 1e-12
        assert np.max(np.abs(vs - ve)) < 1e-6


def test_euler_321_inverts_rot():
    rng = np.random.default_rng(4)
    for _ in range(20):
        v = rng.uniform([-np.pi, -1.4, -np.pi], [np.pi, 1.4, np.pi])
        assert np.allclose(P.euler_321(P.rot(v)), v, atol=1e-13)


def test_planted_target_error_is_not_a_maximum():
    """Taking the farthest point of the feasible circle instead of the nearest
    gives a feasible attitude whose trace a generic optimiser beats."""
    B, J, H = np.asarray(PRM.B), np.asarray(PRM.J), np.asarray(PRM.hmom)
    C = P.reachable_normal(B)
    x0 = np.array([0.1, np.pi / 8, -0.2, 0.05, 0.0, -0.1])
    kappa = -(C @ (J * x0[3:] - P.rot(x0[:3]) @ H)) / np.linalg.norm(H)
    h = H / np.linalg.norm(H)
    p = h - (C @ h) * C
    t = kappa * C - np.sqrt(1 - kappa ** 2) * p / np.linalg.norm(p)   # planted: the far point
    ax = np.cross(h, t)
    s, c = np.linalg.norm(ax), h @ t
    n = ax / s
    K = np.array([[0, -n[2], n[1]], [n[2], 0, -n[0]], [-n[1], n[0], 0]])
    bad = P.euler_321(np.eye(3) + s * K + (1 - c) * K @ K)
    assert abs(-C @ P.rot(bad) @ H - C @ (J * x0[3:] - P.rot(x0[:3]) @ H)) < 1e-12   # still feasible
    vs = _slsqp_target(x0, (x0[:3], np.zeros(3)))
    assert np.trace(P.rot(vs)) > np.trace(P.rot(bad)) + 1e-3
    assert np.max(np.abs(P.target_attitude(PRM, x0) - vs)) < 1e-6
