"""Oracle: closed forms for the linear-quadratic characteristic BVP.

TEST INFRASTRUCTURE ONLY (see oracle/grid.py).

For x' = A x + B u with cost 0.5 int x'Qx + u'Ru + 0.5 x(T)'QT x(T), the
characteristic system of Eq. hamchar is linear, y' = Z y with
Z = [[A, -B R^-1 B'], [-Q, -A']], and lambda(t) = P(t) x(t) where P solves the
Riccati equation.  Over one step of width h the exact flow is M = expm(h Z);
the four-stage Lobatto IIIA collocation step is M = R33(h Z), the (3,3) Pade
approximant of the exponential (the stability function of this collocation
method), R33(z) = p(z) / p(-z) with p(z) = 1 + z/2 + z^2/10 + z^3/120.

Writing M in 6x6 blocks and imposing lambda_i = P_i x_i, lambda_N = QT x_N gives
the backward recursion
    P_i = (M22 - P_{i+1} M12)^{-1} (P_{i+1} M11 - M21),   P_N = QT,
so lambda(0) = P_0 x0.  With M = expm(h Z) this is the continuous Riccati
solution at the mesh points (and V = 0.5 x0' P(0) x0); with M = R33(h Z) it is
the exact root of the collocation equations at the mesh points.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm


def pade33(Zh: np.ndarray) -> np.ndarray:
    I = np.eye(Zh.shape[0])
    Z2 = Zh @ Zh
    Z3 = Z2 @ Zh
    num = I + Zh / 2.0 + Z2 / 10.0 + Z3 / 120.0
    den = I - Zh / 2.0 + Z2 / 10.0 - Z3 / 120.0
    return np.linalg.solve(den, num)


def riccati_p0(prob, T: float, N: int, discrete: bool) -> np.ndarray:
    """P at t = 0 by the backward block recursion over N steps of width T/N."""
    Z = prob.hamiltonian_matrix()
    h = T / N
    M = pade33(h * Z) if discrete else expm(h * Z)
    M11, M12, M21, M22 = M[:6, :6], M[:6, 6:], M[6:, :6], M[6:, 6:]
    P = prob.QT.copy()
    for _ in range(N):
        P = np.linalg.solve(M22 - P @ M12, P @ M11 - M21)
    return P


def lq_lambda0(prob, x0, T, N, discrete=True):
    return riccati_p0(prob, T, N, discrete) @ np.asarray(x0)


def lq_value(prob, x0, T, N=4096):
    """Continuous V(0, x0) = 0.5 x0' P(0) x0."""
    x0 = np.asarray(x0)
    return 0.5 * x0 @ riccati_p0(prob, T, N, discrete=False) @ x0
