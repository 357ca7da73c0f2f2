"""Oracle: Smolyak sparse grids on nested 1-D point sets (Section 3.2).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow FP64 CPU reference
against which the CUDA path is checked.  Only the tests, the smoke check and
the benchmark's CPU-baseline leg may import it; the product never does.

Definitions followed:
  * Nested 1-D sets X^i and increments dX^i = X^i \\ X^{i-1} (Section 3.2).
  * The CGL sets of Eq. CGL: X^1 = {1/2}; X^i = {(1 - cos((k-1) pi / 2^(i-1)))/2,
    k = 1..2^(i-1)+1} for i > 1.
  * The sparse grid G^q = union over |i| <= q of dX^{i_1} x ... x dX^{i_d}.
  * The classic (equispaced, N_1 = 2) and modified (N_1 = 1) sets, used only to
    reproduce the 2-D node counts printed beside Fig. 1 and Fig. 2.

Readings (the paper is garbled or silent here):
  * dN_1 = 1, dN_2 = 2, dN_i = 2^(i-2) for i >= 3 for the CGL and modified sets.
    The bound "1 <= j <= 2^(i-2)" printed for every i > 1 gives dN_2 = 1, which
    reproduces none of the printed node counts.
  * Membership in dX^i is decided by the index k in X^i, never by comparing
    floats: X^(i-1) sits at the odd k of X^i (i >= 3), so dX^i is the even k;
    X^1 = {1/2} is the middle point k = 2 of X^2, so dX^2 is k = 1, 3.  (The
    relation a^i_j = u^i_(2j-1) in the paper is an index garble for CGL.)
  * Node order: by |i|, then i lexicographically, then j lexicographically.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def n_points(i: int, kind: str = "cgl") -> int:
    """|X^i|."""
    if kind == "classic":
        return 2 ** (i - 1) + 1
    return 1 if i == 1 else 2 ** (i - 1) + 1


def cgl_points(i: int) -> np.ndarray:
    """X^i of Eq. CGL on [0, 1].  Evaluated as sin^2(theta/2) = (1 - cos theta)/2,
    which gives exactly 0, 1/2 and 1 at theta = 0, pi/2, pi."""
    if i == 1:
        return np.array([0.5])
    n = 2 ** (i - 1)
    k = np.arange(n + 1)
    theta = k * math.pi / n
    x = np.sin(theta / 2.0) ** 2
    x[0] = 0.0
    x[-1] = 1.0
    if n % 2 == 0:
        x[n // 2] = 0.5
    return x


def delta_k(i: int, kind: str = "cgl") -> list[int]:
    """0-based indices k into X^i of the points of dX^i."""
    if kind == "classic":
        if i == 1:
            return [0, 1]
        return list(range(1, 2 ** (i - 1), 2))
    if i == 1:
        return [0]
    if i == 2:
        return [0, 2]
    return list(range(1, 2 ** (i - 1), 2))


def delta_n(i: int, kind: str = "cgl") -> int:
    return len(delta_k(i, kind))


def multi_indices(d: int, q: int):
    """All i in N^d with i_k >= 1 and |i| <= q, ordered by |i| then lexicographically."""
    out = []
    for s in range(d, q + 1):
        for i in itertools.product(range(1, s - d + 2), repeat=d):
            if sum(i) == s:
                out.append(tuple(i))
    return out


def count_nodes(d: int, q: int, kind: str = "cgl") -> int:
    """|G^q| = sum over |i| <= q of prod dN_{i_k}."""
    return sum(math.prod(delta_n(ik, kind) for ik in i) for i in multi_indices(d, q))


class Grid:
    """A CGL sparse grid on a box.

    Attributes
      d, level (L), q = d + L
      lev   (M, d) int : level i_k of each node in each dimension
      kidx  (M, d) int : 0-based index k of the node's coordinate in X^{i_k}
      unit  (M, d) f64 : coordinates in [0, 1]^d
      x     (M, d) f64 : coordinates mapped to the box lo + (hi - lo) * unit
    """

    def __init__(self, d: int, level: int, lo, hi):
        self.d = d
        self.level = level
        self.q = d + level
        self.lo = np.asarray(lo, dtype=np.float64).copy()
        self.hi = np.asarray(hi, dtype=np.float64).copy()
        lev, kidx = [], []
        for i in multi_indices(d, self.q):
            for ks in itertools.product(*[delta_k(ik) for ik in i]):
                lev.append(i)
                kidx.append(ks)
        self.lev = np.array(lev, dtype=np.int64).reshape(-1, d)
        self.kidx = np.array(kidx, dtype=np.int64).reshape(-1, d)
        self.M = self.lev.shape[0]
        self.unit = np.empty((self.M, d))
        for n in range(self.M):
            for k in range(d):
                self.unit[n, k] = cgl_points(self.lev[n, k])[self.kidx[n, k]]
        self.x = self.lo + (self.hi - self.lo) * self.unit

    def sum_level(self) -> np.ndarray:
        return self.lev.sum(axis=1)

    def fine_key(self, n: int) -> tuple:
        """Position of node n on the finest 1-D set X^(L+1) in every dimension:
        point k of X^i is point k * 2^(L+1-i) of X^(L+1) for i >= 2, and the
        point of X^1 is the middle of X^(L+1)."""
        top = self.level + 1
        key = []
        for k in range(self.d):
            i = self.lev[n, k]
            if i == 1:
                key.append(2 ** (top - 2) if top >= 2 else 0)
            else:
                key.append(int(self.kidx[n, k]) * 2 ** (top - i))
        return tuple(key)
