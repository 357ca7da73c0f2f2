"""Oracle: the optimal control problems and their characteristic equations.

TEST INFRASTRUCTURE ONLY (see oracle/grid.py).

Section 2 defines the Hamiltonian H = L + lambda' f and u* = argmin_u H; the
characteristic BVP of Eq. hamchar is x' = H_lambda', lambda' = -H_x',
z' = L, with x(0) = x0, lambda(T) = grad h(x(T)), z(0) = 0, and Eq. optuv gives
u*(x0) = u*(x0, lambda(0)), V = z(T) + h(x(T)).

Both problems here are control-affine with a quadratic control cost
0.5 u' R u, so u* = -R^{-1} Bf' lambda and, with K = Bf R^{-1} Bf',
    x'      = f0(x) - K lambda
    lambda' = -grad_x l(x) - f0_x(x)' lambda
where l is the state part of the running cost.

Attitude problem (Section 5, Eq. sat_model): x = (v, w), v = (phi, theta, psi)
3-2-1 Euler angles, v' = E(v) w, J w' = S(w) R(v) h + B u.  The paper defers
E, S, R to its reference [kangwilcox]; the reading used here is
  E(v) = [[1, s_phi t_theta, c_phi t_theta], [0, c_phi, -s_phi],
          [0, s_phi / c_theta, c_phi / c_theta]]      (3-2-1 Euler rates),
  R(v) = Rx(phi) Ry(theta) Rz(psi)                   (inertial -> body, R(0) = I),
  S(w) a = a x w                                     (body derivative of a
                                                      constant inertial momentum).
The gradient f0_x' lambda is written out by hand below; a test checks it
against a complex-step derivative of lambda' f0.

LQ problem: f0 = A x, l = 0.5 x'Qx, h = 0.5 x'QT x.
"""
from __future__ import annotations

import numpy as np

import synth


def _mv(A, x):
    """Matrix-vector product, vectorised over trailing point axes of A and/or x."""
    if A.ndim == 2:
        return np.einsum('ij,j...->i...', A, x)
    return np.einsum('ij...,j...->i...', A, x)


def _mm(A, B):
    return np.einsum('ij...,jk...->ik...', A, B)


def _rx(a):
    c, s = np.cos(a), np.sin(a)
    o, z = np.ones_like(a), np.zeros_like(a)
    return np.array([[o, z, z], [z, c, s], [z, -s, c]])


def _ry(a):
    c, s = np.cos(a), np.sin(a)
    o, z = np.ones_like(a), np.zeros_like(a)
    return np.array([[c, z, -s], [z, o, z], [s, z, c]])


def _rz(a):
    c, s = np.cos(a), np.sin(a)
    o, z = np.ones_like(a), np.zeros_like(a)
    return np.array([[c, s, z], [-s, c, z], [z, z, o]])


def _drx(a):
    c, s = np.cos(a), np.sin(a)
    z = np.zeros_like(a)
    return np.array([[z, z, z], [z, -s, c], [z, -c, -s]])


def _dry(a):
    c, s = np.cos(a), np.sin(a)
    z = np.zeros_like(a)
    return np.array([[-s, z, -c], [z, z, z], [c, z, -s]])


def _drz(a):
    c, s = np.cos(a), np.sin(a)
    z = np.zeros_like(a)
    return np.array([[-s, c, z], [-c, -s, z], [z, z, z]])


def rot(v):
    """R(v) = Rx(phi) Ry(theta) Rz(psi)."""
    return _mm(_mm(_rx(v[0]), _ry(v[1])), _rz(v[2]))


def euler_rates(v):
    """E(v) for 3-2-1 angles."""
    ph, th = v[0], v[1]
    sp, cp = np.sin(ph), np.cos(ph)
    ct, tt = np.cos(th), np.tan(th)
    z, o = np.zeros_like(ph), np.ones_like(ph)
    return np.array([[o, sp * tt, cp * tt], [z, cp, -sp], [z, sp / ct, cp / ct]])


def _col(vec, like):
    """A constant 3-vector shaped to broadcast against `like` (3, ...)."""
    return np.asarray(vec).reshape((3,) + (1,) * (like.ndim - 1))


class Attitude:
    """All state arrays are (12, ...) or (6, ...): component first, points after.

    B is 3 x m (m = 3: Example I; m = 2: Example II).  The running cost
    penalises v - v_e for a target attitude v_e (0 unless given; Example II
    takes v_e from target_attitude)."""
    n = 12

    def __init__(self, p: synth.AttitudeParams, target=None):
        self.p = p
        self.Jinv = 1.0 / np.asarray(p.J, dtype=np.float64)
        self.B = np.asarray(p.B, dtype=np.float64)
        self.m = self.B.shape[1]
        self.hmom = np.asarray(p.hmom, dtype=np.float64)
        self.target = np.zeros(3) if target is None else np.asarray(target, dtype=np.float64)
        JB = self.Jinv[:, None] * self.B               # J^{-1} B
        self.Kw = JB @ JB.T / p.r                      # K restricted to the w block

    def f0(self, x):
        v, w = x[:3], x[3:6]
        g = _mv(rot(v), _col(self.hmom, v) * np.ones_like(v))
        return np.concatenate([_mv(euler_rates(v), w),
                               _col(self.Jinv, w) * np.cross(g, w, axis=0)])

    def ustar(self, x, lam):
        """u* = -R^{-1} Bf' lambda with Bf = [0; J^{-1} B], R = r I."""
        return -_mv(self.B.T, _col(self.Jinv, lam) * lam[3:6]) / self.p.r

    def grad_lf0(self, x, lam):
        """grad_x (lambda' f0(x)), written out by hand.

        lambda' f0 = lv' E(v) w + p . (g x w), p = J^{-1} lw, g = R(v) h.
          d/dw   = E(v)' lv + p x g
          d/dv_k = lv' (dE/dv_k) w + (dg/dv_k) . (w x p)
        """
        v, w = x[:3], x[3:6]
        lv, lw = lam[:3], lam[3:6]
        p = _col(self.Jinv, lw) * lw
        ph, th, ps = v
        sp, cp = np.sin(ph), np.cos(ph)
        st, ct = np.sin(th), np.cos(th)
        tt = st / ct
        sec2 = 1.0 / ct ** 2
        E = euler_rates(v)
        z = 0.0 * ph
        dE_dph = np.array([[z, cp * tt, -sp * tt], [z, -sp, -cp], [z, cp / ct, -sp / ct]])
        dE_dth = np.array([[z, sp * sec2, cp * sec2], [z, z, z],
                           [z, sp * st * sec2, cp * st * sec2]])
        Rx, Ry, Rz = _rx(ph), _ry(th), _rz(ps)
        h = _col(self.hmom, v) * np.ones_like(v)
        g = _mv(Rx, _mv(Ry, _mv(Rz, h)))
        dg0 = _mv(_drx(ph), _mv(Ry, _mv(Rz, h)))
        dg1 = _mv(Rx, _mv(_dry(th), _mv(Rz, h)))
        dg2 = _mv(Rx, _mv(Ry, _mv(_drz(ps), h)))
        wxp = np.cross(w, p, axis=0)
        gv = np.stack([(lv * _mv(dE_dph, w)).sum(0) + (dg0 * wxp).sum(0),
                       (lv * _mv(dE_dth, w)).sum(0) + (dg1 * wxp).sum(0),
                       (dg2 * wxp).sum(0)])
        gw = _mv(np.swapaxes(E, 0, 1), lv) + np.cross(p, g, axis=0)
        return np.concatenate([gv, gw])

    def grad_l(self, x):
        return np.concatenate([self.p.wv * (x[:3] - _col(self.target, x[:3])), self.p.ww * x[3:6]])

    def rhs(self, y):
        """Characteristic right-hand side F(y), y = (x, lambda), shape (12, ...)."""
        x, lam = y[:6], y[6:]
        xdot = self.f0(x) - np.concatenate([np.zeros_like(lam[:3]), _mv(self.Kw, lam[3:6])])
        ldot = -self.grad_l(x) - self.grad_lf0(x, lam)
        return np.concatenate([xdot, ldot])

    def running_cost(self, y):
        x, lam = y[:6], y[6:]
        u = self.ustar(x, lam)
        dv = x[:3] - _col(self.target, x[:3])
        return 0.5 * (self.p.wv * (dv ** 2).sum(0) + self.p.ww * (x[3:6] ** 2).sum(0)
                      + self.p.r * (u ** 2).sum(0))

    def terminal(self, x):
        return 0.5 * (self.p.tv * (x[:3] ** 2).sum(0) + self.p.tw * (x[3:6] ** 2).sum(0))

    def terminal_grad(self, x):
        return np.concatenate([self.p.tv * x[:3], self.p.tw * x[3:6]])

    def terminal_hess(self, x):
        return np.diag(np.concatenate([np.full(3, self.p.tv), np.full(3, self.p.tw)]))

    def hamiltonian(self, y):
        """H*(x, lambda) = L(x, u*) + lambda' f(x, u*)."""
        x, lam = y[:6], y[6:]
        u = self.ustar(x, lam)
        Bu = _mv(self.B, u)
        f = self.f0(x) + np.concatenate([np.zeros_like(Bu), _col(self.Jinv, Bu) * Bu])
        return self.running_cost(y) + (lam * f).sum(0)


class LinearQuadratic:
    n = 12
    m = 3

    def __init__(self, p: synth.LQParams):
        self.p = p
        self.A = np.asarray(p.A, dtype=np.float64)
        self.B = np.asarray(p.B, dtype=np.float64)
        self.Q = np.asarray(p.Q, dtype=np.float64)
        self.R = np.asarray(p.R, dtype=np.float64)
        self.QT = np.asarray(p.QT, dtype=np.float64)
        self.Rinv = np.linalg.inv(self.R)
        self.K = self.B @ self.Rinv @ self.B.T

    def f0(self, x):
        return _mv(self.A, x)

    def ustar(self, x, lam):
        return -_mv(self.Rinv @ self.B.T, lam)

    def rhs(self, y):
        x, lam = y[:6], y[6:]
        return np.concatenate([_mv(self.A, x) - _mv(self.K, lam),
                               -_mv(self.Q, x) - _mv(self.A.T, lam)])

    def running_cost(self, y):
        x, lam = y[:6], y[6:]
        u = self.ustar(x, lam)
        return 0.5 * ((x * _mv(self.Q, x)).sum(0) + (u * _mv(self.R, u)).sum(0))

    def terminal(self, x):
        return 0.5 * (x * _mv(self.QT, x)).sum(0)

    def terminal_grad(self, x):
        return _mv(self.QT, x)

    def terminal_hess(self, x):
        return self.QT

    def hamiltonian(self, y):
        x, lam = y[:6], y[6:]
        u = self.ustar(x, lam)
        return self.running_cost(y) + (lam * (_mv(self.A, x) + _mv(self.B, u))).sum(0)

    def hamiltonian_matrix(self):
        """Z with y' = Z y: [[A, -B R^-1 B'], [-Q, -A']]."""
        return np.block([[self.A, -self.K], [-self.Q, -self.A.T]])


class Example3:
    """Example III of Section 5: three states in components 0..2 of the
    six-state layout (components 3..5 have zero dynamics and cost), one
    control entering x3' through B(x) = g e3, g = 1 + x1^2 + x2^2;
    l(x) = 0.5 x3^2 / g^2, L = l + 0.5 u^2, no terminal cost.
    u* = -g lambda3 and H* = l + lambda' f0 - 0.5 g^2 lambda3^2, so
        x'      = f0(x) - g^2 lambda3 e3
        lambda' = -(grad l + grad_x(lambda' f0) - g lambda3^2 grad g)."""
    n = 12
    m = 1

    def __init__(self, p=None):
        self.p = p

    @staticmethod
    def _g(x):
        return 1.0 + x[0] ** 2 + x[1] ** 2

    def f0(self, x):
        x1, x2, x3 = x[0], x[1], x[2]
        g = self._g(x)
        q = -2 * x1 ** 2 + 2 * x1 * x2 - 2 * x2 ** 2 + 2 * x2 * x3 / g
        z = 0.0 * x1
        return np.stack([-x1 + x2, -x2 + x3 / g, q * x3 / g, z, z, z])

    def ustar(self, x, lam):
        return (-self._g(x) * lam[2])[None, ...] if np.ndim(lam[2]) else np.array([-self._g(x) * lam[2]])

    def grad_lf0(self, x, lam):
        """grad_x (lambda' f0(x)), written out by hand (a test checks it
        against a complex-step derivative)."""
        x1, x2, x3 = x[0], x[1], x[2]
        l1, l2, l3 = lam[0], lam[1], lam[2]
        g = self._g(x)
        q = -2 * x1 ** 2 + 2 * x1 * x2 - 2 * x2 ** 2 + 2 * x2 * x3 / g
        dq1 = -4 * x1 + 2 * x2 - 4 * x1 * x2 * x3 / g ** 2
        dq2 = 2 * x1 - 4 * x2 + 2 * x3 / g - 4 * x2 ** 2 * x3 / g ** 2
        dq3 = 2 * x2 / g
        df2 = (-2 * x1 * x3 / g ** 2, -1 - 2 * x2 * x3 / g ** 2, 1 / g)
        df3 = (x3 * (dq1 / g - 2 * x1 * q / g ** 2), x3 * (dq2 / g - 2 * x2 * q / g ** 2), q / g + x3 * dq3 / g)
        z = 0.0 * x1
        return np.stack([-l1 + l2 * df2[0] + l3 * df3[0],
                         l1 + l2 * df2[1] + l3 * df3[1],
                         l2 * df2[2] + l3 * df3[2], z, z, z])

    def grad_l(self, x):
        x1, x2, x3 = x[0], x[1], x[2]
        g = self._g(x)
        z = 0.0 * x1
        return np.stack([-2 * x1 * x3 ** 2 / g ** 3, -2 * x2 * x3 ** 2 / g ** 3, x3 / g ** 2, z, z, z])

    def rhs(self, y):
        x, lam = y[:6], y[6:]
        g = self._g(x)
        z = 0.0 * g
        xdot = self.f0(x) - np.stack([z, z, g ** 2 * lam[2], z, z, z])
        gradg = np.stack([2 * x[0], 2 * x[1], z, z, z, z])
        ldot = -(self.grad_l(x) + self.grad_lf0(x, lam) - g * lam[2] ** 2 * gradg)
        return np.concatenate([xdot, ldot])

    def running_cost(self, y):
        x, lam = y[:6], y[6:]
        g = self._g(x)
        return 0.5 * (x[2] ** 2 / g ** 2 + (g * lam[2]) ** 2)

    def terminal(self, x):
        return 0.0 * x[0]

    def terminal_grad(self, x):
        return 0.0 * x

    def terminal_hess(self, x):
        return np.zeros((6, 6))

    def hamiltonian(self, y):
        x, lam = y[:6], y[6:]
        g = self._g(x)
        u = -g * lam[2]
        f = self.f0(x)
        return self.running_cost(y) + (lam * f).sum(0) + lam[2] * g * u

    @staticmethod
    def value(tau, x):
        """The closed form printed with Example III: V = 0.5 x3^2 / g^2 tanh(tau),
        tau = T - t the remaining horizon."""
        g = 1.0 + x[0] ** 2 + x[1] ** 2
        return 0.5 * x[2] ** 2 / g ** 2 * np.tanh(tau)

    @staticmethod
    def feedback(tau, x):
        """u* = -x3 / g tanh(tau) (printed with Example III)."""
        g = 1.0 + x[0] ** 2 + x[1] ** 2
        return -x[2] / g * np.tanh(tau)


def reachable_normal(B):
    """C with C' B = 0 (Example II: the momentum direction the wheels cannot
    change), unit length; for m = 2 the cross product of B's columns."""
    B = np.asarray(B, dtype=np.float64)
    c = np.cross(B[:, 0], B[:, 1])
    return c / np.linalg.norm(c)


def euler_321(R):
    """The angles v = (phi, theta, psi) with rot(v) = R, |theta| < pi/2.
    From R = Rx(phi) Ry(theta) Rz(psi): R[0, 2] = -sin theta,
    R[0, :2] = cos theta (cos psi, sin psi), R[1:, 2] = cos theta (sin phi, cos phi)."""
    return np.array([np.arctan2(R[1, 2], R[2, 2]), -np.arcsin(R[0, 2]), np.arctan2(R[0, 1], R[0, 0])])


def target_attitude(params, x0):
    """Eq. optim_attitude: v_e = argmax tr R(v) subject to
    -C' R(v) H = C' (J w0 - R(v0) H), x0 = (v0, w0); NaN when no rotation
    satisfies the constraint.

    Solved in closed form from the geometry of rotations, not by an iterative
    optimiser.  tr R = 1 + 2 cos(a), a the rotation angle of R, so the maximum
    is the rotation of smallest angle in the feasible set.  The constraint
    fixes the component along C of the body-frame vector R h, h = H / |H|:
    C' R h = kappa = -C' (J w0 - R(v0) H) / |H|.  A rotation taking h to a unit
    vector t turns through at least the angle between h and t, and the turn
    about h x t attains it.  So the optimum takes h to the point t of the
    circle {t : |t| = 1, C't = kappa} nearest to h, which lies in the plane of
    C and h:  t = kappa C + sqrt(1 - kappa^2) p / |p|,  p = h - (C'h) C,
    and R is the rotation about h x t by the angle between h and t
    (Rodrigues' formula).  v_e are its 3-2-1 angles."""
    B = np.asarray(params.B, dtype=np.float64)
    J = np.asarray(params.J, dtype=np.float64)
    H = np.asarray(params.hmom, dtype=np.float64)
    C = reachable_normal(B)
    v0, w0 = np.asarray(x0[:3], dtype=np.float64), np.asarray(x0[3:6], dtype=np.float64)
    kappa = -(C @ (J * w0 - rot(v0) @ H)) / np.linalg.norm(H)
    if not abs(kappa) <= 1.0:
        return np.full(3, np.nan)
    h = H / np.linalg.norm(H)
    p = h - (C @ h) * C
    t = kappa * C + np.sqrt(1.0 - kappa * kappa) * p / np.linalg.norm(p)
    axis = np.cross(h, t)
    s, c = np.linalg.norm(axis), h @ t
    if s == 0.0:
        return np.zeros(3) if c > 0 else np.full(3, np.nan)
    n = axis / s
    K = np.array([[0.0, -n[2], n[1]], [n[2], 0.0, -n[0]], [-n[1], n[0], 0.0]])
    R = np.eye(3) + s * K + (1.0 - c) * (K @ K)   # sin a = s, cos a = c
    return euler_321(R)


def make(params, target=None):
    if params.kind == synth.ATTITUDE:
        return Attitude(params, target)
    if params.kind == synth.EXAMPLE3:
        return Example3(params)
    return LinearQuadratic(params)


def rhs_jacobian(prob, y, eps: float = 1e-30):
    """dF/dy by complex-step differentiation of F: column c is
    Im F(y + i eps e_c) / eps, exact to rounding for real-analytic F.
    y is (12, ...); the result is (12, 12, ...)."""
    n = y.shape[0]
    J = np.empty((n, n) + y.shape[1:])
    for c in range(n):
        yc = y.astype(np.complex128)
        yc[c] = yc[c] + 1j * eps
        J[:, c] = prob.rhs(yc).imag / eps
    return J
