"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module only draws numbers: problem parameters (momentum vector, control
matrix, linear system matrices), query states and per-node horizons.  It holds
none of the method's arithmetic (no grid, no basis, no BVP, no interpolant), so
the oracle and the CUDA path can both take their inputs from here without
sharing any computation.

Workloads follow the 6-D rigid-body / momentum-wheel attitude problem of
Section 5 (Example I) and a 6-D linear-quadratic problem used as a closed-form
check.  Seeds default to 0 for problem data and 1 for queries.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ATTITUDE = 0
LQ = 1
EXAMPLE3 = 2

BOX_HALF = np.pi / 4.0


@dataclass
class AttitudeParams:
    """Parameters of the attitude problem (Section 5, Eq. sat_model).

    State x = (phi, theta, psi, w1, w2, w3).  Running cost
    0.5*(wv*|v|^2 + ww*|w|^2 + r*|u|^2), terminal cost
    0.5*(tv*|v(T)|^2 + tw*|w(T)|^2).
    """
    J: np.ndarray                      # (3,) diagonal inertia
    hmom: np.ndarray                   # (3,) total angular momentum (inertial frame)
    B: np.ndarray                      # (3,3) control matrix
    wv: float = 1.0
    ww: float = 1.0
    r: float = 0.1
    tv: float = 1.0
    tw: float = 1.0
    kind: int = field(default=ATTITUDE, init=False)
    # B may be 3 x m (m = 2: Example II's two pairs of wheels); the running cost
    # then penalises v - v_e with a per-state target v_e (Example II)


@dataclass
class LQParams:
    """Linear-quadratic problem x' = A x + B u, cost 0.5 x'Qx + 0.5 u'Ru, terminal 0.5 x'QT x."""
    A: np.ndarray   # (6,6)
    B: np.ndarray   # (6,3)
    Q: np.ndarray   # (6,6)
    R: np.ndarray   # (3,3)
    QT: np.ndarray  # (6,6)
    kind: int = field(default=LQ, init=False)


@dataclass
class Example3Params:
    """Example III of Section 5 (three states, one control, no parameters).
    The value function is interpolated on a (t, x) grid over
    t in [0, 5], x in [-2, 2]^3; the horizon of a node at time t is
    t_end - t.  The final time is not printed; t_end = 10 is the reading
    (with any t_end >= 7 the interpolation error of the exact V on the q = 12
    grid matches the printed mean 8.5e-4 and variance 2.8e-6)."""
    t_end: float = 10.0
    kind: int = field(default=EXAMPLE3, init=False)


def example3_params() -> Example3Params:
    return Example3Params()


def example3_box():
    """The (t, x1, x2, x3) region D of Example III: [0, 5] x [-2, 2]^3."""
    return np.array([0.0, -2.0, -2.0, -2.0]), np.array([5.0, 2.0, 2.0, 2.0])


def example3_mesh(horizon, h: float = 5.0 / 32.0):
    """Intervals per node for horizons t_end - t: the mesh width closest to h
    from above (at least one interval; a zero horizon keeps one)."""
    return np.maximum(1, np.ceil(np.asarray(horizon) / h - 1e-9)).astype(np.int32)


def attitude_params(seed: int = 0) -> AttitudeParams:
    """Synthetic attitude problem shaped like Example I: J = diag(2,3,4),
    |h| = 1 seeded, B = I + U(-0.1,0.1) off-diagonal, reseeded until cond(B) < 10."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(3)
    hmom = g / np.linalg.norm(g)
    while True:
        B = np.eye(3) + rng.uniform(-0.1, 0.1, size=(3, 3)) * (1.0 - np.eye(3))
        if np.linalg.cond(B) < 10.0:
            break
    return AttitudeParams(J=np.array([2.0, 3.0, 4.0]), hmom=hmom, B=B)


def example1_params() -> AttitudeParams:
    """The printed parameters of Example I (Section 5.1): B, J, H = (1,1,1),
    W1 = W2 = 1, W3 = 1/2, terminal W4|v|^2 + W5|w|^2 with W4 = W5 = 1
    (no factor 1/2, so the terminal weights in the 0.5*t*|.|^2 form are 2)."""
    B = np.array([[1.0, 1.0 / 20.0, 1.0 / 10.0],
                  [1.0 / 15.0, 1.0, 1.0 / 10.0],
                  [1.0 / 10.0, 1.0 / 15.0, 1.0]])
    return AttitudeParams(J=np.array([2.0, 3.0, 4.0]), hmom=np.ones(3), B=B,
                          wv=1.0, ww=1.0, r=0.5, tv=2.0, tw=2.0)


def example2_params() -> AttitudeParams:
    """The printed parameters of Example II (Section 5): two pairs of momentum
    wheels, B = [[1, 1/10], [0, 1], [1/12, 0]], J = diag(2, 3, 4),
    H = (12, 12, 6), L = W1/2 |v - v_e|^2 + W2/2 |w|^2 + W3/2 |u|^2 with
    W1 = 1, W2 = 2, W3 = 0.5, no terminal cost, T = 30."""
    B = np.array([[1.0, 0.1], [0.0, 1.0], [1.0 / 12.0, 0.0]])
    return AttitudeParams(J=np.array([2.0, 3.0, 4.0]), hmom=np.array([12.0, 12.0, 6.0]), B=B,
                          wv=1.0, ww=2.0, r=0.5, tv=0.0, tw=0.0)


EXAMPLE2_T = 30.0


def example2_box():
    """The domain D of Example II: v in [-pi/6, pi/6]^3, w in [-pi/8, pi/8]^3."""
    return (np.array([-np.pi / 6] * 3 + [-np.pi / 8] * 3), np.array([np.pi / 6] * 3 + [np.pi / 8] * 3))


def lq_params(seed: int = 0) -> LQParams:
    """Seeded 6-D LQ problem: A = A0 - (alpha(A0) + 0.1) I with A0 ~ N(0,1),
    so the spectral abscissa of A is -0.1; B ~ N(0,1) 6x3; Q = I, R = 0.1 I, QT = I."""
    rng = np.random.default_rng(seed)
    A0 = rng.standard_normal((6, 6))
    alpha = np.max(np.linalg.eigvals(A0).real)
    A = A0 - (alpha + 0.1) * np.eye(6)
    B = rng.standard_normal((6, 3))
    return LQParams(A=A, B=B, Q=np.eye(6), R=0.1 * np.eye(3), QT=np.eye(6))


def box(d: int = 6, half: float = BOX_HALF):
    """Symmetric box [-half, half]^d as (lo, hi)."""
    return -half * np.ones(d), half * np.ones(d)


def uniform_queries(n: int, lo, hi, seed: int = 1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return lo + (hi - lo) * rng.random((n, lo.size))


def mixed_queries(n: int, lo, hi, sigma: float = 0.2, seed: int = 1) -> np.ndarray:
    """Half uniform on the box, half N(0, sigma^2 I) clipped to the box."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    nu = n // 2
    u = lo + (hi - lo) * rng.random((nu, lo.size))
    g = np.clip(sigma * rng.standard_normal((n - nu, lo.size)), lo, hi)
    q = np.concatenate([u, g], axis=0)
    return q[rng.permutation(n)]


def mixed_horizons(n: int, seed: int = 2):
    """Per-node horizon T drawn from {10, 20, 40}, with mesh N = 6.4 T intervals
    (64 / 128 / 256), i.e. one mesh width h = 5/32 for all."""
    rng = np.random.default_rng(seed)
    T = rng.choice(np.array([10.0, 20.0, 40.0]), size=n)
    N = np.rint(6.4 * T).astype(np.int32)
    return T, N
