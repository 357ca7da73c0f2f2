"""Pins of the oracle's sparse grid and interpolant against what the paper and
the mathematics fix (node counts, nestedness, the Kronecker property, exact
reproduction of the Smolyak polynomial space, the combination formula, and the
Theorem 1 bound)."""
import math
import os

import numpy as np
import pytest

import synth
from oracle import grid as G
from oracle import interp as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


@pytest.mark.parametrize("row", _rows("node_counts.txt"), ids=lambda r: f"{r[0]}-d{r[1]}-q{r[2]}")
def test_node_counts(row):
    kind, d, q, count = row[0], int(row[1]), int(row[2]), int(row[3])
    assert G.count_nodes(d, q, kind) == count


def test_enumerated_grid_matches_count_and_is_unique():
    for L in range(0, 4):
        g = G.Grid(6, L, *synth.box())
        assert g.M == G.count_nodes(6, 6 + L)
        keys = {g.fine_key(n) for n in range(g.M)}
        assert len(keys) == g.M
        assert np.unique(np.round(g.unit, 14), axis=0).shape[0] == g.M


def test_cgl_sets_nested_and_symmetric():
    for i in range(2, 9):
        x = G.cgl_points(i)
        assert x.size == G.n_points(i)
        assert np.allclose(x + x[::-1], 1.0, atol=1e-15)
        coarse = G.cgl_points(i - 1)
        if i >= 3:
            assert np.allclose(x[::2], coarse, atol=1e-15)
        # the increment points are exactly the ones not in the coarser set
        new = x[G.delta_k(i)]
        for p in new:
            assert np.min(np.abs(coarse - p)) > 1e-6
    assert G.cgl_points(2).tolist() == [0.0, 0.5, 1.0]


def test_node_zero_is_centre_and_grid_symmetric():
    g = G.Grid(6, 3, *synth.box())
    assert np.all(g.x[0] == 0.0)
    pts = {tuple(np.round(r, 12)) for r in g.x}
    for r in g.x:
        assert tuple(np.round(-r, 12) + 0.0) in pts


def test_basis_kronecker_property():
    for i in range(1, 7):
        X = G.cgl_points(i)
        for k in G.delta_k(i):
            vals = I.basis_1d(i, k, X)
            expect = np.zeros(X.size)
            expect[k] = 1.0
            assert np.allclose(vals, expect, atol=1e-13)
            # a^i_j vanishes on every coarser set
            for i2 in range(1, i):
                assert np.allclose(I.basis_1d(i, k, G.cgl_points(i2)), 0.0, atol=1e-13)


@pytest.fixture(scope="module")
def grid2():
    return G.Grid(6, 2, *synth.box())


def test_interpolant_exact_at_nodes(grid2):
    f = np.random.default_rng(3).standard_normal((grid2.M, 3))
    w = I.surpluses(grid2, f)
    assert np.allclose(I.eval_surplus(grid2, w, grid2.x), f, atol=1e-13, rtol=0)


def _unit_poly(g, exps):
    def f(x):
        u = (np.atleast_2d(x) - g.lo) / (g.hi - g.lo)
        return np.prod([u[:, k] ** e for k, e in enumerate(exps)], axis=0)
    return f


@pytest.mark.parametrize("exps", [(2, 2, 0, 0, 0, 0), (4, 0, 0, 0, 0, 0), (3, 0, 0, 0, 0, 0),
                                  (0, 2, 0, 0, 0, 1), (1, 0, 0, 0, 0, 0)])
def test_reproduces_smolyak_space(grid2, exps):
    # x^e with e <= N_{i}-1 in each direction for some |i| <= q lies in the space
    f = _unit_poly(grid2, exps)
    w = I.surpluses(grid2, f(grid2.x))
    xq = synth.uniform_queries(40, grid2.lo, grid2.hi, seed=7)
    assert np.max(np.abs(I.eval_surplus(grid2, w, xq) - f(xq))) <= 1e-13


@pytest.mark.parametrize("exps", [(5, 0, 0, 0, 0, 0), (2, 2, 2, 0, 0, 0), (1, 1, 1, 0, 0, 0)])
def test_does_not_reproduce_outside_space(grid2, exps):
    f = _unit_poly(grid2, exps)
    w = I.surpluses(grid2, f(grid2.x))
    xq = synth.uniform_queries(40, grid2.lo, grid2.hi, seed=7)
    assert np.max(np.abs(I.eval_surplus(grid2, w, xq) - f(xq))) > 1e-6


def test_surplus_form_equals_combination_form():
    g = G.Grid(6, 2, *synth.box())
    f = np.random.default_rng(5).standard_normal((g.M, 2))
    w = I.surpluses(g, f)
    xq = synth.mixed_queries(30, g.lo, g.hi, seed=9)
    a = I.eval_surplus(g, w, xq)
    b = I.eval_combination(g, f, xq)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


def test_surplus_form_equals_combination_form_3d_level4():
    g = G.Grid(3, 4, -np.ones(3), 2 * np.ones(3))
    f = np.random.default_rng(6).standard_normal(g.M)
    w = I.surpluses(g, f)
    xq = synth.uniform_queries(30, g.lo, g.hi, seed=2)
    assert np.allclose(I.eval_surplus(g, w, xq), I.eval_combination(g, f, xq), atol=1e-11)


def test_theorem1_bound_reproduced():
    """Eq. ebvpbound with Lambda_i from Eq. lebesgue at N = 2^(i-1) (Lambda_1 = 1)
    gives the printed bound 3.66e4 at q = 13, d = 6 (to the printed 3 digits,
    about 0.3%)."""
    d, q, printed = _rows("theorem1_bound.txt")[0]
    d, q, printed = int(d), int(q), float(printed)
    gam = 0.5772156649015329

    def lam(i):
        if i == 1:
            return 1.0
        n = 2 ** (i - 1)
        return (2 / math.pi) * (math.log(n) + gam + math.log(4 / math.pi) + math.log(2))

    total = 0.0
    for l in range(q - d + 1, q + 1):
        s_l = sum(math.prod(lam(ik) for ik in i) for i in G.multi_indices(d, l) if sum(i) == l)
        total += math.comb(d - 1, q - l) * s_l
    assert abs(total - printed) / printed < 3e-3
