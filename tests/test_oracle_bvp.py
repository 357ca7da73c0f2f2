"""Pins of the oracle's characteristic-BVP solver: the Lobatto IIIA tableau,
the problem definitions, the Riccati closed forms of the LQ case, Hamiltonian
constancy, PMP/HJB consistency, and the equilibrium at the origin."""
import os

import numpy as np
import pytest

import synth
from oracle import bvp, lobatto, riccati
from oracle import problems as P

GOLD = os.path.join(os.path.dirname(__file__), "golden")
S5 = np.sqrt(5.0)


# ---------------------------------------------------------------- tableau
def test_lobatto_tableau_textbook_values():
    """Four-stage Lobatto IIIA coefficients in closed form (Hairer & Wanner,
    Solving ODEs II, Table IV.5.7)."""
    A, b, c = lobatto.tableau()
    A_ref = np.array([
        [0, 0, 0, 0],
        [(11 + S5) / 120, (25 - S5) / 120, (25 - 13 * S5) / 120, (-1 + S5) / 120],
        [(11 - S5) / 120, (25 + 13 * S5) / 120, (25 + S5) / 120, (-1 - S5) / 120],
        [1 / 12, 5 / 12, 5 / 12, 1 / 12]])
    assert np.allclose(A, A_ref, atol=4e-15, rtol=0)
    assert np.allclose(c, [0, (5 - S5) / 10, (5 + S5) / 10, 1], atol=1e-15)
    assert np.allclose(b, [1 / 12, 5 / 12, 5 / 12, 1 / 12], atol=4e-15)


def test_lobatto_order_conditions():
    A, b, c = lobatto.tableau()
    for m in range(1, 7):                      # quadrature order 2s-2 = 6
        assert abs(b @ c ** (m - 1) - 1.0 / m) < 1e-14
    for m in range(1, 5):                      # stage order s = 4
        assert np.allclose(A @ c ** (m - 1), c ** m / m, atol=1e-14)


def test_lobatto_stability_is_pade33():
    A, b, _ = lobatto.tableau()
    for z in [-3.0, -0.5, 0.1, 1.7, 2.5 + 1.0j]:
        R = 1.0 + z * b @ np.linalg.solve(np.eye(4) - z * A, np.ones(4))
        p = lambda s: 1 + s / 2 + s ** 2 / 10 + s ** 3 / 120
        assert abs(R - p(z) / p(-z)) < 1e-13 * abs(R)


# ---------------------------------------------------------------- problems
@pytest.fixture(scope="module")
def att():
    return P.make(synth.attitude_params())


@pytest.fixture(scope="module")
def lq():
    return P.make(synth.lq_params())


def test_costate_gradient_matches_complex_step(att):
    y = np.random.default_rng(0).uniform(-0.8, 0.8, size=(12, 7))
    x, lam = y[:6], y[6:]
    g = att.grad_lf0(x, lam)
    cs = np.zeros_like(g)
    for k in range(6):
        xc = x.astype(complex)
        xc[k] = xc[k] + 1e-30j
        cs[k] = (lam * att.f0(xc)).sum(0).imag / 1e-30
    assert np.allclose(g, cs, atol=1e-14, rtol=1e-13)


def test_costate_equation_is_minus_hamiltonian_gradient(att):
    """lambda' = -dH*/dx and x' = dH*/dlambda (Eq. hamchar), by complex step of H*."""
    y = np.random.default_rng(1).uniform(-0.8, 0.8, size=12)
    F = att.rhs(y[:, None])[:, 0]
    dH = np.zeros(12)
    for k in range(12):
        yc = y.astype(complex)
        yc[k] += 1e-30j
        dH[k] = att.hamiltonian(yc[:, None]).imag[0] / 1e-30
    assert np.allclose(F[:6], dH[6:], atol=1e-13)
    assert np.allclose(F[6:], -dH[:6], atol=1e-13)


def test_rhs_jacobian_matches_central_differences(att, lq):
    for pr in (att, lq):
        y = np.random.default_rng(2).uniform(-0.7, 0.7, size=(12, 3))
        J = P.rhs_jacobian(pr, y)
        eps = 1e-6
        for c in range(12):
            yp, ym = y.copy(), y.copy()
            yp[c] += eps
            ym[c] -= eps
            fd = (pr.rhs(yp) - pr.rhs(ym)) / (2 * eps)
            assert np.allclose(J[:, c], fd, atol=1e-7)


def test_rotation_and_euler_rate_kinematics(att):
    """R(v) is a rotation with R(0) = I, and v' = E(v) w is the 3-2-1 Euler-rate
    map of the body rate w: dR/dt = -[w]x R for R inertial -> body."""
    rng = np.random.default_rng(4)
    assert np.allclose(P.rot(np.zeros(3)), np.eye(3))
    for _ in range(5):
        v = rng.uniform(-1.0, 1.0, 3)
        w = rng.uniform(-1.0, 1.0, 3)
        R = P.rot(v)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1.0) < 1e-14
        vdot = P.euler_rates(v) @ w
        eps = 1e-6
        Rdot = (P.rot(v + eps * vdot) - P.rot(v - eps * vdot)) / (2 * eps)
        wx = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
        assert np.allclose(Rdot, -wx @ R, atol=1e-8)


def test_body_momentum_is_rotated_constant(att):
    """S(w) R(v) h = d/dt (R(v) h) along v' = E(v) w: the gyroscopic term is the
    body-frame derivative of a constant inertial momentum."""
    rng = np.random.default_rng(5)
    v = rng.uniform(-1.0, 1.0, 3)
    w = rng.uniform(-1.0, 1.0, 3)
    x = np.concatenate([v, w])
    eps = 1e-6
    vdot = P.euler_rates(v) @ w
    d = (P.rot(v + eps * vdot) @ att.hmom - P.rot(v - eps * vdot) @ att.hmom) / (2 * eps)
    assert np.allclose(att.f0(x[:, None])[3:, 0], att.Jinv * d, atol=1e-8)


# ---------------------------------------------------------------- LQ closed forms
X0_LQ = np.array([0.5, -0.3, 0.2, 0.7, -0.1, 0.4])


@pytest.mark.parametrize("T,N", [(1.0, 4), (2.0, 16), (10.0, 128)])
def test_lq_newton_one_step_and_discrete_riccati(lq, T, N):
    """The collocation root at the mesh points is the Pade(3,3) Riccati recursion.
    Short horizons matter: once P(t) reaches the algebraic Riccati solution, any
    A-stable rational step gives the same lambda(0), so only T = 1, 2 tell the
    discrete map apart (from the exponential by ~5e-7 at T = 1, N = 4)."""
    s = bvp.solve(lq, X0_LQ, T, N)
    assert s.status == bvp.CONVERGED and s.iters == 1
    ref = riccati.lq_lambda0(lq, X0_LQ, T, N, discrete=True)
    assert np.max(np.abs(s.lambda0 - ref)) <= 1e-12 * np.max(np.abs(ref))
    if T == 1.0:
        cont = riccati.lq_lambda0(lq, X0_LQ, T, N, discrete=False)
        assert np.max(np.abs(cont - ref)) > 1e-7 * np.max(np.abs(ref))


def test_lq_continuous_riccati_on_fine_mesh(lq):
    s = bvp.solve(lq, X0_LQ, 10.0, 1024)
    lam = riccati.lq_lambda0(lq, X0_LQ, 10.0, 1024, discrete=False)
    V = riccati.lq_value(lq, X0_LQ, 10.0)
    assert np.max(np.abs(s.lambda0 - lam)) <= 1e-8 * np.max(np.abs(lam))
    assert abs(s.V - V) <= 1e-8 * abs(V)


def test_lq_feedback_linear_in_state(lq):
    """u*(x0) = -R^-1 B' P(0) x0 is linear in x0."""
    a = bvp.solve(lq, X0_LQ, 10.0, 32)
    b = bvp.solve(lq, 2.0 * X0_LQ, 10.0, 32)
    assert np.allclose(b.u0, 2.0 * a.u0, rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------- attitude
X0_ATT = (np.pi / 4) * np.array([1, -1, 1, -1, 1, 1])


def test_origin_is_equilibrium(att):
    s = bvp.solve(att, np.zeros(6), 20.0, 64)
    assert s.status == bvp.CONVERGED and s.iters == 0
    assert s.V == 0.0 and np.all(s.lambda0 == 0.0) and np.all(s.Y == 0.0)


def test_hamiltonian_constant_along_solution(att):
    """H* is constant along optimal trajectories of a time-invariant problem;
    the collocation solution keeps it to O(h^p), p >= 4."""
    devs = []
    for N in (32, 64, 128):
        s = bvp.solve(att, X0_ATT, 20.0, N)
        assert s.status == bvp.CONVERGED
        H = att.hamiltonian(s.Y.T)
        devs.append(H.max() - H.min())
    assert devs[0] / devs[1] > 2 ** 4 and devs[1] / devs[2] > 2 ** 4
    assert devs[2] < 1e-5


def test_value_gradient_is_initial_costate(att):
    """PMP/HJB consistency: dV/dx0 = lambda(0)."""
    N, eps = 128, 1e-4
    s = bvp.solve(att, X0_ATT, 20.0, N)
    g = np.array([(bvp.solve(att, X0_ATT + eps * e, 20.0, N).V
                   - bvp.solve(att, X0_ATT - eps * e, 20.0, N).V) / (2 * eps) for e in np.eye(6)])
    assert np.max(np.abs(g - s.lambda0)) < 1e-6


def test_residual_recomputed_at_root(att):
    s = bvp.solve(att, 0.5 * X0_ATT, 10.0, 64)
    F = bvp.residual(att, s.Y, 0.5 * X0_ATT, 10.0, 64)
    assert np.max(np.abs(F)) <= 1e-12 and s.resid <= 1e-12


def test_newton_correction_lands_on_the_root(att, lq):
    """The Newton step that bounds the distance of an iterate to the root:
    on the linear problem one step from any iterate lands on the root; on the
    attitude problem the step from Y* + delta cancels delta to second order."""
    Y0 = bvp.initial_guess(X0_LQ, 16) + np.random.default_rng(0).standard_normal((49, 12))
    root = bvp.solve(lq, X0_LQ, 2.0, 16).Y
    D = bvp.newton_correction(lq, Y0, X0_LQ, 2.0, 16)
    assert np.max(np.abs(Y0 + D - root)) <= 1e-11 * np.max(np.abs(root))
    s = bvp.solve(att, 0.5 * X0_ATT, 10.0, 32)
    delta = np.random.default_rng(1).standard_normal(s.Y.shape)
    errs = []
    for eps in (1e-4, 5e-5):
        Yp = s.Y + eps * delta
        D = bvp.newton_correction(att, Yp, 0.5 * X0_ATT, 10.0, 32)
        assert np.max(np.abs(D + eps * delta)) <= 1e-2 * eps          # D ~ -delta
        errs.append(np.max(np.abs(Yp + D - s.Y)))
    assert errs[0] / errs[1] > 3.0                                       # quadratic


def test_example1_sign_and_scale():
    """Example I worked trajectory (Fig. Trajectories): the printed u(0).  The
    paper defers E, S, R to another reference; with the reading used here the
    solve reproduces the signs and the scale of u(0) but not its digits
    (u2 differs by 40%), so the convention is recorded as unpinned and only
    this loose check is made."""
    vals = {}
    with open(os.path.join(GOLD, "example1_trajectory.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    x0 = np.array([vals[k] for k in ("phi0", "theta0", "psi0", "w1_0", "w2_0", "w3_0")])
    u_ref = np.array([vals["u1_0"], vals["u2_0"], vals["u3_0"]])
    pr = P.make(synth.example1_params())
    s = bvp.solve(pr, x0, 20.0, 64, polish=False)
    assert s.status == bvp.CONVERGED
    assert np.all(np.sign(s.u0) == np.sign(u_ref))
    assert np.max(np.abs(s.u0 - u_ref)) < 0.5 * np.max(np.abs(u_ref))


# ---------------------------------------------------------------- planted mistakes
def test_pins_catch_a_sign_error_in_the_costate_equation(att, monkeypatch):
    """A flipped gyroscopic term in grad_x(lambda' f0) breaks the Hamiltonian
    structure, which the Hamiltonian-gradient pin detects."""
    orig = P.Attitude.grad_lf0

    def broken(self, x, lam):
        g = orig(self, x, lam)
        g[3:] = g[3:] - 2 * np.cross(self.Jinv[:, None] * lam[3:6], P._mv(P.rot(x[:3]), self.hmom[:, None] * np.ones_like(x[:3])), axis=0)
        return g

    monkeypatch.setattr(P.Attitude, "grad_lf0", broken)
    y = np.random.default_rng(1).uniform(-0.8, 0.8, size=12)
    F = att.rhs(y[:, None])[:, 0]
    dH = np.zeros(12)
    for k in range(12):
        yc = y.astype(complex)
        yc[k] += 1e-30j
        dH[k] = att.hamiltonian(yc[:, None]).imag[0] / 1e-30
    assert not np.allclose(F[6:], -dH[:6], atol=1e-6)


def test_pins_catch_a_wrong_tableau_entry(lq, monkeypatch):
    """A perturbed Lobatto coefficient moves the LQ root off the Pade-Riccati value."""
    A = bvp._A.copy()
    A[2, 1] += 1e-3
    monkeypatch.setattr(bvp, "_A", A)
    s = bvp.solve(lq, X0_LQ, 1.0, 4)
    ref = riccati.lq_lambda0(lq, X0_LQ, 1.0, 4, discrete=True)
    assert np.max(np.abs(s.lambda0 - ref)) > 1e-6 * np.max(np.abs(ref))
