"""Oracle pins for Example III (Section 5): the closed-form value function
and feedback printed with the example, the hand-written gradient against a
complex step, the characteristic equations against the Hamiltonian, and the
zero horizon.  A planted mistake in the costate equation must fail the
closed-form pin."""
import numpy as np
import pytest

import synth
from oracle import bvp
from oracle import problems as P

PR = P.make(synth.example3_params())
CASES = [(5.0, (0.5, -0.3, 1.2)), (2.0, (-1.5, 1.0, -0.7)), (0.5, (2.0, 2.0, 2.0)),
         (3.7, (-2.0, 0.4, 1.9)), (1.0, (0.0, 0.0, -1.3))]


def _x(x3):
    x = np.zeros(6)
    x[:3] = x3
    return x


@pytest.mark.parametrize("tau,x3", CASES)
def test_closed_form_value_and_feedback(tau, x3):
    """V(t, x) = 0.5 x3^2 / g^2 tanh(T - t), u* = -x3 / g tanh(T - t): the
    Lobatto IIIA solution on a 5/32-wide mesh agrees to the discretisation
    error (order 6)."""
    N = max(1, int(np.ceil(tau / (5 / 32))))
    s = bvp.solve(PR, _x(x3), tau, N, tol=1e-12)
    assert s.status == bvp.CONVERGED
    x = np.array(x3)
    assert abs(s.V - P.Example3.value(tau, x)) <= 1e-7 * max(1.0, abs(P.Example3.value(tau, x)))
    assert abs(s.u0[0] - P.Example3.feedback(tau, x)) <= 1e-6
    g = 1 + x[0] ** 2 + x[1] ** 2
    assert abs(s.lambda0[2] - x[2] / g ** 2 * np.tanh(tau)) <= 1e-6
    assert np.allclose(s.lambda0[3:], 0.0) and np.allclose(s.Y[:, 3:6], 0.0)


def test_discretisation_error_is_sixth_order():
    x, tau = np.array([0.5, -0.3, 1.2]), 5.0
    e = [abs(bvp.solve(PR, _x(x), tau, N, tol=1e-13).V - P.Example3.value(tau, x)) for N in (8, 16)]
    assert e[0] / e[1] > 2 ** 5


def test_grad_lf0_matches_complex_step():
    rng = np.random.default_rng(3)
    for _ in range(5):
        x, lam = _x(rng.uniform(-2, 2, 3)), np.concatenate([rng.standard_normal(3), np.zeros(3)])
        gs = np.empty(6)
        for c in range(6):
            xc = x.astype(np.complex128)
            xc[c] += 1e-30j
            gs[c] = (lam * PR.f0(xc)).sum().imag / 1e-30
        assert np.allclose(PR.grad_lf0(x, lam), gs, rtol=1e-13, atol=1e-13)


def test_characteristics_are_hamiltonian_gradients():
    """x' = dH*/dlambda and lambda' = -dH*/dx, by complex step of H*."""
    rng = np.random.default_rng(4)
    y = np.concatenate([rng.uniform(-2, 2, 3), np.zeros(3), rng.standard_normal(3), np.zeros(3)])
    dH = np.empty(12)
    for c in range(12):
        yc = y.astype(np.complex128)
        yc[c] += 1e-30j
        dH[c] = PR.hamiltonian(yc).imag / 1e-30
    F = PR.rhs(y)
    assert np.allclose(F[:6], dH[6:], atol=1e-12) and np.allclose(F[6:], -dH[:6], atol=1e-12)


def test_zero_horizon():
    s = bvp.solve(PR, _x((1.0, -1.0, 0.5)), 0.0, 1, tol=1e-12)
    assert s.status == bvp.CONVERGED and s.V == 0.0 and np.all(s.lambda0 == 0.0) and s.u0[0] == 0.0


def test_planted_sign_error_fails_closed_form():
    class Wrong(P.Example3):
        def rhs(self, y):
            F = super().rhs(y)
            x, lam = y[:6], y[6:]
            g = self._g(x)
            F[6] += 2 * g * lam[2] ** 2 * 2 * x[0]   # flips the sign of the g lambda3^2 grad g term
            return F
    tau, x = 2.0, np.array([-1.5, 1.0, -0.7])
    s = bvp.solve(Wrong(), _x(x), tau, 13, tol=1e-12)
    assert abs(s.u0[0] - P.Example3.feedback(tau, x)) > 1e-4
