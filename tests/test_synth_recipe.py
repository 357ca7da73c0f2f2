"""The seeded input recipe both sides share: shapes, distributions and the
structure the benchmark workload is stated to have (pure numpy, no GPU)."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import synth  # noqa: E402


def test_attitude_parameters_match_the_stated_model():
    p = synth.attitude_params(0)
    assert np.allclose(np.diag(p.J) if np.ndim(p.J) == 2 else p.J, [2.0, 3.0, 4.0])
    assert abs(np.linalg.norm(p.hmom) - 1.0) <= 1e-15
    # the cost of the stated model: 0.5 (|v|^2 + |w|^2 + 0.1 |u|^2), terminal 0.5 (|v|^2 + |w|^2)
    assert (p.wv, p.ww, p.r, p.tv, p.tw) == (1.0, 1.0, 0.1, 1.0, 1.0)
    B = np.asarray(p.B)
    assert B.shape == (3, 3) and np.linalg.cond(B) < 10.0
    assert np.allclose(np.diag(B), 1.0) and np.all(np.abs(B - np.eye(3)) <= 0.1)
    # the same seed gives the same problem, another seed another one
    q = synth.attitude_params(0)
    assert np.array_equal(np.asarray(q.B), B) and np.array_equal(q.hmom, p.hmom)
    assert not np.array_equal(np.asarray(synth.attitude_params(1).B), B)


def test_mixed_queries_half_uniform_half_clipped_gaussian():
    lo, hi = synth.box(6)
    n = 200_000
    q = synth.mixed_queries(n, lo, hi, seed=3)
    assert q.shape == (n, 6) and np.all(q >= lo) and np.all(q <= hi)
    assert np.array_equal(q, synth.mixed_queries(n, lo, hi, seed=3))
    # the two halves, in the generator's order before any shuffling: compare moments
    # of the whole set with the mixture's (uniform variance (2a)^2/12, Gaussian 0.04)
    a = hi[0]
    var_mix = 0.5 * (2 * a) ** 2 / 12 + 0.5 * 0.2 ** 2   # clipping at pi/4 ~ 3.9 sigma is negligible
    assert abs(q.var(axis=0).mean() - var_mix) <= 0.01 * var_mix
    assert abs(q.mean()) <= 5e-3
    # the Gaussian half puts about half the mass inside |x| < 0.2 beyond the uniform share
    inside = np.mean(np.abs(q[:, 0]) < 0.2)
    expect = 0.5 * (0.4 / (2 * a)) + 0.5 * 0.6827
    assert abs(inside - expect) <= 0.01


def test_mixed_horizons_pair_T_with_one_mesh_width():
    T, N = synth.mixed_horizons(1457, seed=2)
    assert set(np.unique(T)) == {10.0, 20.0, 40.0}
    assert np.all(N == np.rint(6.4 * T)) and set(np.unique(N)) == {64, 128, 256}
    assert np.allclose(T / N, 5.0 / 32.0)
    # roughly uniform over the three horizons
    counts = np.array([np.sum(T == t) for t in (10.0, 20.0, 40.0)])
    assert np.all(np.abs(counts - 1457 / 3) <= 4 * np.sqrt(1457 * (1 / 3) * (2 / 3)))
