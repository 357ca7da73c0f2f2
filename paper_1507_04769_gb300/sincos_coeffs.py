"""Coefficients of the FP64 sine and cosine polynomials on |x| <= pi/4 used by
the right-hand side kernels (`dsincos` in csrc/problems.cuh).

With z = x^2 the kernels evaluate
    sin x = x + x z P(z),        P of degree SIN_DEG,
    cos x = 1 - z/2 + z^2 Q(z),  Q of degree COS_DEG,
by Horner's rule with fused multiply-adds.  P and Q are the weighted minimax
approximations, on 0 <= z <= (pi/4)^2, of
    g_s(z) = (sin(sqrt z)/sqrt z - 1)/z   with weight  z sqrt(z)/sin(sqrt z),
    g_c(z) = (cos(sqrt z) - 1 + z/2)/z^2  with weight  z^2/cos(sqrt z),
i.e. they minimise the largest relative error of sin and cos themselves.  They
are found by the Remez exchange algorithm (E. Ya. Remez, 1934): solve for the
polynomial whose weighted error equioscillates on a reference set of
degree + 2 points, move the reference to the extrema of that error, repeat.
Arithmetic in mpmath at 60 digits; the coefficients are then rounded to
doubles and the error of the rounded polynomials is measured again.

This module is run by hand to print the coefficients (python -m
paper_1507_04769_gb300.sincos_coeffs) and by a test that checks the kernel's
literals against it.  It is not imported by the library at run time.
"""
from __future__ import annotations

import functools

import mpmath as mp

SIN_DEG = 5
COS_DEG = 5


def _targets():
    zmax = (mp.pi / 4) ** 2

    def gs(z):
        if z == 0:
            return mp.mpf(-1) / 6
        x = mp.sqrt(z)
        return (mp.sin(x) / x - 1) / z

    def ws(z):
        if z == 0:
            return mp.mpf(0)
        x = mp.sqrt(z)
        return z * x / mp.sin(x)

    def gc(z):
        if z == 0:
            return mp.mpf(1) / 24
        x = mp.sqrt(z)
        return (mp.cos(x) - 1 + z / 2) / z ** 2

    def wc(z):
        return z ** 2 / mp.cos(mp.sqrt(z))

    return zmax, (gs, ws), (gc, wc)


def _peval(c, z):
    acc = mp.mpf(0)
    for a in reversed(c):
        acc = acc * z + a
    return acc


def remez(g, w, deg: int, zmax, iters: int = 30, grid: int = 4000):
    """Weighted minimax polynomial of degree `deg` for g on [0, zmax]: the
    coefficients (lowest first) and the levelled weighted error."""
    n = deg + 2
    # initial reference: Chebyshev extrema mapped to [0, zmax]
    ref = [zmax * (1 - mp.cos(mp.pi * i / (n - 1))) / 2 for i in range(n)]
    ref[0] = zmax * mp.mpf("1e-6")   # the weight vanishes at 0
    c, E = None, None
    zs = [zmax * mp.mpf(i) / grid for i in range(1, grid + 1)]
    for _ in range(iters):
        A = mp.matrix(n, n)
        b = mp.matrix(n, 1)
        for i, z in enumerate(ref):
            for j in range(deg + 1):
                A[i, j] = z ** j
            A[i, deg + 1] = (-1) ** i / w(z)
            b[i] = g(z)
        sol = mp.lu_solve(A, b)
        c = [sol[j] for j in range(deg + 1)]
        E = sol[deg + 1]
        err = [w(z) * (_peval(c, z) - g(z)) for z in zs]
        # local extrema of the error with alternating signs, n of them
        ext = []
        for i in range(len(zs)):
            lo = err[i - 1] if i > 0 else None
            hi = err[i + 1] if i + 1 < len(zs) else None
            e = err[i]
            is_ext = (lo is None or abs(e) >= abs(lo)) and (hi is None or abs(e) >= abs(hi))
            if is_ext and (not ext or mp.sign(e) != mp.sign(ext[-1][1])):
                ext.append((zs[i], e))
            elif is_ext and abs(e) > abs(ext[-1][1]):
                ext[-1] = (zs[i], e)
        while len(ext) > n:   # drop the smallest end
            if abs(ext[0][1]) < abs(ext[-1][1]):
                ext.pop(0)
            else:
                ext.pop()
        if len(ext) < n:
            break
        new_ref = [z for z, _ in ext]
        if max(abs(a - b) for a, b in zip(new_ref, ref)) < zmax * mp.mpf("1e-12"):
            ref = new_ref
            break
        ref = new_ref
    return c, abs(E)


def rounded_error(c_double, g, w, zmax, samples: int = 20000) -> float:
    """Largest weighted error of the polynomial with double coefficients,
    measured in high precision (no evaluation rounding)."""
    c = [mp.mpf(v) for v in c_double]
    worst = mp.mpf(0)
    for i in range(1, samples + 1):
        z = zmax * mp.mpf(i) / samples
        worst = max(worst, abs(w(z) * (_peval(c, z) - g(z))))
    return float(worst)


@functools.lru_cache(maxsize=1)
def coefficients():
    """(P, Q) as lists of Python floats, lowest degree first, with the
    largest relative error of sin and cos from each rounded polynomial."""
    with mp.workdps(60):
        zmax, (gs, ws), (gc, wc) = _targets()
        cs, _ = remez(gs, ws, SIN_DEG, zmax)
        cc, _ = remez(gc, wc, COS_DEG, zmax)
        P = [float(v) for v in cs]
        Q = [float(v) for v in cc]
        return P, Q, rounded_error(P, gs, ws, zmax), rounded_error(Q, gc, wc, zmax)


if __name__ == "__main__":
    P, Q, es, ec = coefficients()
    print(f"sin: relative error of the rounded polynomial {es:.3e}")
    for j, v in enumerate(P):
        print(f"  P[{j}] = {v.hex()}  ({v!r})")
    print(f"cos: relative error of the rounded polynomial {ec:.3e}")
    for j, v in enumerate(Q):
        print(f"  Q[{j}] = {v.hex()}  ({v!r})")
