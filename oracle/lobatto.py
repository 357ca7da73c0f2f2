"""Oracle: the four-stage Lobatto IIIA collocation tableau (Section 3.1).

TEST INFRASTRUCTURE ONLY (see oracle/grid.py).

The BVP solver of the paper is the four-point Lobatto IIIA collocation formula
(Section 3.1, after Kierzenka and Shampine).  Its abscissae are the Gauss-Lobatto
points of [0, 1], the roots of x(1-x) P3'(2x-1): c = 0, (5 - sqrt5)/10,
(5 + sqrt5)/10, 1, and its coefficients are the collocation conditions
a_kj = integral from 0 to c_k of the Lagrange polynomial l_j on c, b_j = a_4j.
They are computed here from that definition with numpy polynomials.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import polynomial as P


def abscissae() -> np.ndarray:
    # roots of the derivative of the degree-3 Legendre polynomial, mapped to [0,1]
    leg3 = np.polynomial.legendre.Legendre.basis(3)
    inner = np.sort(leg3.deriv().roots().real)
    return np.concatenate([[0.0], (inner + 1.0) / 2.0, [1.0]])


def tableau():
    """(A, b, c) of the 4-stage Lobatto IIIA method."""
    c = abscissae()
    s = c.size
    A = np.zeros((s, s))
    for j in range(s):
        # Lagrange polynomial l_j on the abscissae, power-basis coefficients
        coef = np.array([1.0])
        for m in range(s):
            if m != j:
                coef = P.polymul(coef, np.array([-c[m], 1.0]) / (c[j] - c[m]))
        integ = P.polyint(coef)
        for k in range(s):
            A[k, j] = P.polyval(c[k], integ) - P.polyval(0.0, integ)
    b = A[-1].copy()
    return A, b, c
