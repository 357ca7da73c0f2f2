"""Oracle: the characteristic BVP at one initial state, Lobatto IIIA + Newton.

TEST INFRASTRUCTURE ONLY (see oracle/grid.py).

Discretisation (Section 3.1, Eq. hamchar): the horizon [0, T] is cut into N
equal intervals of width h = T/N.  On interval i the four Lobatto IIIA stages
Y_{i,1} = y_i, Y_{i,2}, Y_{i,3}, Y_{i,4} = y_{i+1} satisfy
    Y_{i,k} - y_i - h sum_j a_kj F(Y_{i,j}) = 0,   k = 2, 3, 4,
with F the characteristic right-hand side.  The unknowns are the 3N+1 distinct
points (y_0, Y_{0,2}, Y_{0,3}, y_1, ..., y_N), each in R^12.  Boundary rows:
x(0) - x0 = 0 and lambda(T) - grad h(x(T)) = 0.  Unknowns and equations are
12(3N+1) each.

Newton (readings; the paper names only the collocation formula):
  * Jacobian of the whole uncondensed system, assembled from complex-step 12x12
    blocks, solved by LAPACK's banded LU with partial pivoting
    (scipy.linalg.solve_banded).  This is deliberately a different linear
    algebra from the CUDA path (stage condensation + block elimination).
  * Damping: Armijo backtracking on 0.5 |F|_2^2, alpha in {1, 1/2, ..., 2^-10},
    sufficient decrease |F(Y + a D)|^2 <= (1 - 2e-4 a) |F(Y)|^2; if no alpha
    passes, the smallest is taken.
  * Converged when |F|_inf <= tol (default 1e-8); stage rows are in y units,
    boundary rows raw.  For parity checks the iteration then continues until
    |F|_inf <= 1e-13 or it stops shrinking, so the answer is the discrete root
    to about 1e-14.
  * Initial guess ("zero control"): lambda = 0 (so u* = 0) and x held at x0 on
    every point.  Integrating the uncontrolled dynamics instead drives the
    Euler angles through theta = +-pi/2 over T = 20, where E(v) is singular.

Outputs (Eq. optuv): lambda(0), u*(x0) = u*(x0, lambda(0)), and
V = z(T) + h(x(T)) where z(T) = h sum_i sum_j b_j L(Y_{i,j}) is the Lobatto
IIIA step applied to z' = L, z(0) = 0.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.linalg import solve_banded

from . import lobatto
from .problems import rhs_jacobian

CONVERGED, MAXITER, NONFINITE, SINGULAR = 0, 1, 2, 3

_A, _B, _C = lobatto.tableau()


@dataclass
class Solution:
    Y: np.ndarray          # (3N+1, 12)
    lambda0: np.ndarray    # (6,)
    u0: np.ndarray         # (m,)
    V: float
    iters: int             # Newton iterations until |F|_inf <= tol
    status: int
    resid: float           # |F|_inf at the returned Y


def initial_guess(x0, N):
    Y = np.zeros((3 * N + 1, 12))
    Y[:, :6] = np.asarray(x0, dtype=np.float64)
    return Y


def residual(prob, Y, x0, T, N):
    """Stacked residual: [x(0)-x0 (6); per interval stages 2,3,4 (36); lambda(T)-grad h (6)]."""
    h = T / N
    F = prob.rhs(Y.T).T                          # (3N+1, 12)
    out = np.empty(12 * (3 * N + 1))
    out[:6] = Y[0, :6] - x0
    for i in range(N):
        p = 3 * i
        for k in range(1, 4):
            r = Y[p + k] - Y[p] - h * (_A[k, 0] * F[p] + _A[k, 1] * F[p + 1]
                                       + _A[k, 2] * F[p + 2] + _A[k, 3] * F[p + 3])
            row = 6 + 36 * i + 12 * (k - 1)
            out[row:row + 12] = r
    xT, lT = Y[-1, :6], Y[-1, 6:]
    out[-6:] = lT - prob.terminal_grad(xT)
    return out


LBW = UBW = 41   # lower / upper bandwidth of the uncondensed Jacobian


def jacobian_banded(prob, Y, T, N):
    """The residual Jacobian in LAPACK band storage ab[UBW + r - c, c]."""
    n = 12 * (3 * N + 1)
    h = T / N
    Jp = rhs_jacobian(prob, Y.T)                # (12, 12, 3N+1)
    ab = np.zeros((LBW + UBW + 1, n))
    I12 = np.eye(12)

    def put(r0, c0, blk):
        rr, cc = np.indices(blk.shape)
        ab[UBW + r0 + rr - (c0 + cc), c0 + cc] = blk

    put(0, 0, np.hstack([np.eye(6), np.zeros((6, 6))]))
    for i in range(N):
        p = 3 * i
        for k in range(1, 4):
            row = 6 + 36 * i + 12 * (k - 1)
            for j in range(4):
                blk = -h * _A[k, j] * Jp[:, :, p + j]
                if j == 0:
                    blk = blk - I12
                if j == k:
                    blk = blk + I12
                put(row, 12 * (p + j), blk)
    xT = Y[-1, :6]
    put(n - 6, n - 12, np.hstack([-prob.terminal_hess(xT), np.eye(6)]))
    return ab


def outputs(prob, Y, T, N):
    h = T / N
    Lc = prob.running_cost(Y.T)                  # (3N+1,)
    z = 0.0
    for i in range(N):
        p = 3 * i
        z += h * (_B[0] * Lc[p] + _B[1] * Lc[p + 1] + _B[2] * Lc[p + 2] + _B[3] * Lc[p + 3])
    V = z + prob.terminal(Y[-1, :6])
    lam0 = Y[0, 6:].copy()
    u0 = prob.ustar(Y[0, :6], lam0)
    return lam0, u0, V


def newton_correction(prob, Y, x0, T, N):
    """The full Newton step D = -J(Y)^-1 F(Y) at an iterate Y, shape (3N+1, 12).
    Near a root Y* of the collocation system, Y + D - Y* = O(|Y - Y*|^2), so
    |D| measures how far Y is from the discrete root (used to bound the error
    of a solve stopped at a residual tolerance)."""
    F = residual(prob, Y, x0, T, N)
    D = solve_banded((LBW, UBW), jacobian_banded(prob, Y, T, N), -F)
    return D.reshape(Y.shape)


def solve(prob, x0, T, N, tol=1e-8, max_iter=50, polish=True, Y0=None):
    """Newton on the full collocation system.  Returns a Solution."""
    x0 = np.asarray(x0, dtype=np.float64)
    Y = initial_guess(x0, N) if Y0 is None else np.array(Y0, dtype=np.float64)
    F = residual(prob, Y, x0, T, N)
    it = 0
    status = MAXITER
    iters_to_tol = -1
    extra = 0
    while True:
        fin = np.max(np.abs(F))
        if not np.isfinite(fin):
            status = NONFINITE
            break
        if fin <= tol and iters_to_tol < 0:
            iters_to_tol = it
            status = CONVERGED
            if not polish:
                break
        if iters_to_tol >= 0:
            if fin <= 1e-13 or extra >= 6:
                break
        if it >= max_iter:
            break
        ab = jacobian_banded(prob, Y, T, N)
        try:
            D = solve_banded((LBW, UBW), ab, -F)
        except np.linalg.LinAlgError:
            status = SINGULAR
            break
        f2 = F @ F
        alpha = 1.0
        while True:
            Yt = Y + alpha * D.reshape(Y.shape)
            Ft = residual(prob, Yt, x0, T, N)
            if np.all(np.isfinite(Ft)) and Ft @ Ft <= (1.0 - 2e-4 * alpha) * f2:
                break
            if alpha <= 2.0 ** -10:
                break
            alpha *= 0.5
        if iters_to_tol >= 0:
            # polishing: stop once the residual no longer shrinks
            if not np.max(np.abs(Ft)) < 0.5 * fin:
                if np.max(np.abs(Ft)) < fin:
                    Y, F = Yt, Ft
                break
            extra += 1
        Y, F = Yt, Ft
        it += 1
    lam0, u0, V = outputs(prob, Y, T, N)
    return Solution(Y=Y, lambda0=lam0, u0=u0, V=V,
                    iters=iters_to_tol if iters_to_tol >= 0 else it,
                    status=status, resid=float(np.max(np.abs(F))))


def solve_many(prob, X0, T, N, **kw):
    """Independent solves at every row of X0 (one BVP per node, Section 3)."""
    X0 = np.atleast_2d(X0)
    T = np.broadcast_to(np.asarray(T, dtype=np.float64), (X0.shape[0],))
    N = np.broadcast_to(np.asarray(N), (X0.shape[0],))
    return [solve(prob, X0[n], float(T[n]), int(N[n]), **kw) for n in range(X0.shape[0])]
