"""Oracle: hierarchical sparse-grid interpolation (Section 3.3).

TEST INFRASTRUCTURE ONLY (see oracle/grid.py).

  * basis_1d: a^i_j, the Lagrange polynomial on all of X^i that is 1 at its
    point of dX^i and 0 at the other points of X^i, written as the literal
    product formula of Section 3.3.  a^1_1 = 1 (Lagrange polynomial on one point).
  * surpluses: Eq. interpo.  I^{d-1} = 0 and, level by level for q' = d..q,
    w = f(x) - I^{q'-1}(f)(x) at every node with |i| = q'.
  * eval_surplus: I^q(f)(x) = sum of w times the tensor product of a^{i_k}_{j_k}.
  * eval_combination: Eq. interpolation2, the combination formula over full
    tensor Lagrange interpolants U^{i_1} x ... x U^{i_d}; an independent route to
    the same polynomial, used as the oracle's self-check.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from .grid import Grid, cgl_points, multi_indices


def lagrange(nodes: np.ndarray, k: int, x) -> np.ndarray:
    """Lagrange polynomial on `nodes` that is 1 at nodes[k]; product formula."""
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    for m, xm in enumerate(nodes):
        if m != k:
            out = out * (x - xm) / (nodes[k] - xm)
    return out


def basis_1d(i: int, k: int, x) -> np.ndarray:
    """a^i at the point k of X^i (k 0-based index into X^i)."""
    x = np.asarray(x, dtype=np.float64)
    if i == 1:
        return np.ones_like(x)
    return lagrange(cgl_points(i), k, x)


def basis_table(grid: Grid, unit_pts: np.ndarray) -> np.ndarray:
    """Phi[p, n] = prod_k a^{lev[n,k]}_{kidx[n,k]}(unit_pts[p, k]) for points in [0,1]^d."""
    unit_pts = np.atleast_2d(unit_pts)
    P = unit_pts.shape[0]
    phi = np.ones((P, grid.M))
    # one 1-D evaluation per distinct (dimension, level, index)
    for k in range(grid.d):
        cache = {}
        for n in range(grid.M):
            key = (grid.lev[n, k], grid.kidx[n, k])
            if key not in cache:
                cache[key] = basis_1d(key[0], key[1], unit_pts[:, k])
            phi[:, n] *= cache[key]
    return phi


def to_unit(grid: Grid, x: np.ndarray) -> np.ndarray:
    return (np.atleast_2d(x) - grid.lo) / (grid.hi - grid.lo)


def surpluses(grid: Grid, f: np.ndarray) -> np.ndarray:
    """Hierarchical surpluses of values f (M, k) at the grid nodes, Eq. interpo."""
    f = np.asarray(f, dtype=np.float64)
    squeeze = f.ndim == 1
    f = f.reshape(grid.M, -1)
    w = np.zeros_like(f)
    s = grid.sum_level()
    phi = basis_table(grid, grid.unit)          # phi[n, m] = basis of node m at node n
    for qq in range(grid.d, grid.q + 1):
        new = np.nonzero(s == qq)[0]
        old = np.nonzero(s < qq)[0]
        # I^{qq-1}(f) at the new nodes uses only surpluses of coarser levels
        interp_prev = phi[np.ix_(new, old)] @ w[old] if old.size else 0.0
        w[new] = f[new] - interp_prev
    return w[:, 0] if squeeze else w


def eval_surplus(grid: Grid, w: np.ndarray, xq: np.ndarray) -> np.ndarray:
    """I^q(f)(xq) = sum over nodes of w_n prod_k a(x_k)."""
    phi = basis_table(grid, to_unit(grid, xq))
    return phi @ w


def eval_combination(grid: Grid, f: np.ndarray, xq: np.ndarray) -> np.ndarray:
    """I^q(f)(xq) by Eq. interpolation2.

    For each i with q-d+1 <= |i| <= q, the full tensor Lagrange interpolant on
    X^{i_1} x ... x X^{i_d} is weighted by (-1)^(q-|i|) C(d-1, q-|i|).  Every
    point of such a tensor grid is a sparse-grid node; it is looked up by its
    position on the finest 1-D set."""
    f = np.asarray(f, dtype=np.float64)
    squeeze = f.ndim == 1
    f = f.reshape(grid.M, -1)
    d, q, top = grid.d, grid.q, grid.level + 1
    lookup = {grid.fine_key(n): n for n in range(grid.M)}
    u = to_unit(grid, xq)
    out = np.zeros((u.shape[0], f.shape[1]))

    def fine_pos(i, k):
        if i == 1:
            return 2 ** (top - 2) if top >= 2 else 0
        return k * 2 ** (top - i)

    for i in multi_indices(d, q):
        s = sum(i)
        if s < q - d + 1:
            continue
        coef = (-1) ** (q - s) * math.comb(d - 1, q - s)
        # 1-D Lagrange values u^{i_k}_k on all of X^{i_k}
        vals = []
        for kk, ik in enumerate(i):
            pts = cgl_points(ik)
            vals.append(np.stack([lagrange(pts, m, u[:, kk]) if ik > 1 else np.ones(u.shape[0])
                                  for m in range(pts.size)], axis=1))
        for ks in itertools.product(*[range(cgl_points(ik).size) for ik in i]):
            node = lookup[tuple(fine_pos(ik, kk) for ik, kk in zip(i, ks))]
            prod = np.ones(u.shape[0])
            for kk in range(d):
                prod = prod * vals[kk][:, ks[kk]]
            out += coef * prod[:, None] * f[node][None, :]
    return out[:, 0] if squeeze else out
