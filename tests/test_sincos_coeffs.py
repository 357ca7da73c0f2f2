"""The FP64 sine/cosine polynomials of the right-hand side kernels: the literals
in csrc/problems.cuh are the rounded Remez minimax coefficients derived by
sincos_coeffs.py, and that derivation meets its error target.  The GPU test
test_library_sincos_within_few_ulp measures the compiled evaluation against
numpy."""
import os
import re

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

from paper_1507_04769_gb300 import sincos_coeffs as sc  # noqa: E402

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_1507_04769_gb300", "csrc", "problems.cuh")


def _kernel_literals():
    text = open(SRC).read()
    body = text[text.index("void dsincos(double a"):]
    body = body[:body.index("sincos(a, s, c);")]
    lits = [float.fromhex(h) for h in re.findall(r"-?0x[0-9a-f]\.[0-9a-f]+p[-+]?\d+", body)]
    # P from degree 5 down to 0, then Q from degree 5 down to 0
    return lits[:6][::-1], lits[6:12][::-1]


def test_kernel_literals_are_the_minimax_coefficients():
    P, Q, es, ec = sc.coefficients()
    kP, kQ = _kernel_literals()
    assert kP == P and kQ == Q
    # the rounded polynomials are well inside one unit in the last place
    eps = np.finfo(np.float64).eps
    assert es < 0.1 * eps and ec < 0.1 * eps


def test_polynomials_equioscillate_below_the_taylor_error():
    """Independent of the fit: the polynomials' largest relative error on
    [-pi/4, pi/4], sampled at 2001 points in 40-digit arithmetic, is below
    that of the Taylor polynomials of the same degree (a plausible fitting
    mistake, a wrong sign or a dropped term, makes it far larger)."""
    P, Q, _, _ = sc.coefficients()
    mp.mp.dps = 40
    xs = [mp.mpf(i) / 1000 * mp.pi / 4 for i in range(-1000, 1001) if i != 0]

    def worst(fs, fc):
        ws = wc = mp.mpf(0)
        for x in xs:
            z = x * x
            ws = max(ws, abs((x + x * z * fs(z)) / mp.sin(x) - 1))
            wc = max(wc, abs((1 + z * (mp.mpf(-0.5) + z * fc(z))) / mp.cos(x) - 1))
        return float(ws), float(wc)

    def horner(c):
        return lambda z: sum(mp.mpf(a) * z ** j for j, a in enumerate(c))

    taylor_P = [(-1) ** (j + 1) / mp.factorial(2 * j + 3) for j in range(6)]
    taylor_Q = [(-1) ** j / mp.factorial(2 * j + 4) for j in range(6)]
    ms, mc = worst(horner(P), horner(Q))
    ts, tc = worst(horner(taylor_P), horner(taylor_Q))
    assert ms < 1.5e-17 and mc < 1e-18
    assert ms < ts and mc < tc
