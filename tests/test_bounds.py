"""Error amplification of the interpolant (Section 4.2): the library's
Theorem 1 factor (host arithmetic, no GPU) against the printed bound and
independent evaluations, and the Monte-Carlo estimate on the GPU."""
import math
import os

import numpy as np
import pytest

from oracle import grid as G

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _sg():
    from paper_1507_04769_gb300 import sg
    return sg


def _lam(i):
    if i == 1:
        return 1.0
    n = 2 ** (i - 1)
    return (2 / math.pi) * (math.log(n) + 0.5772156649015329 + math.log(4 / math.pi) + math.log(2))


def test_theorem1_bound_matches_printed_value():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "theorem1_bound.txt")) if l.strip() and l[0] != "#"]
    d, q, printed = int(rows[0][0]), int(rows[0][1]), float(rows[0][2])
    b = _sg().theorem1_bound(d, q)
    assert abs(b - printed) / printed < 3e-3


@pytest.mark.parametrize("d,q", [(2, 5), (3, 6), (4, 7), (6, 9)])
def test_theorem1_bound_by_enumeration(d, q):
    """S_l by explicit enumeration of the multi-indices (oracle's enumerator)."""
    total = 0.0
    for l in range(q - d + 1, q + 1):
        s_l = sum(math.prod(_lam(k) for k in i) for i in G.multi_indices(d, l) if sum(i) == l)
        total += math.comb(d - 1, q - l) * s_l
    assert abs(_sg().theorem1_bound(d, q) - total) <= 1e-12 * total


def test_theorem1_bound_one_dimension_is_the_lebesgue_bound():
    for q in range(1, 12):
        assert abs(_sg().theorem1_bound(1, q) - _lam(q)) <= 1e-14 * _lam(q)


def test_theorem1_bound_rejects_bad_arguments():
    sg = _sg()
    for d, q in ((0, 3), (3, 2), (65, 70)):
        with pytest.raises(sg.SGError):
            sg.theorem1_bound(d, q)


@pytest.mark.gpu
def test_mc_error_amplification_below_theorem1_bound():
    """q = 13, d = 6 (44,689 nodes), 2,000 points as in Section 4.2 (the paper
    reports 66.60 for its sample): the estimate lies between the largest
    nodal value and the Theorem 1 bound."""
    sg = _sg()
    est = sg.mc_error_amplification(6, 7, 2000, seed=0)
    assert 0.5 < est < sg.theorem1_bound(6, 13)
    sym = sg.mc_error_amplification(6, 7, 2000, seed=0, symmetric=True)
    assert 0.5 < sym < sg.theorem1_bound(6, 13)
