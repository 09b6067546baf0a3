"""Pins of the oracle's farthest-point anchor selection (oracle/anchors.py):
a closed form, the factor-2 guarantee of the greedy k-center rule against a
brute-force optimum, and the invariants of its output."""

import itertools

import numpy as np
import pytest

from oracle import anchors as oa


def _line(m):
    return np.stack([np.arange(m, dtype=np.float64), np.zeros(m), np.zeros(m)], axis=1)


def test_collinear_points_give_dyadic_subdivisions():
    xyz = _line(17)
    assert oa.farthest_point(xyz, 2).tolist() == [0, 16]
    assert oa.farthest_point(xyz, 3).tolist() == [0, 8, 16]
    # 4 and 12 are equally far: the lower index joins first
    assert oa.farthest_point(xyz, 4).tolist() == [0, 4, 8, 16]
    assert oa.farthest_point(xyz, 5).tolist() == [0, 4, 8, 12, 16]
    assert oa.farthest_point(xyz, 9).tolist() == list(range(0, 17, 2))
    assert oa.farthest_point(xyz, 17).tolist() == list(range(17))
    # from the middle: both ends tie, the lower index first
    assert oa.farthest_point(xyz, 2, start=8).tolist() == [0, 8]
    assert oa.farthest_point(xyz, 3, start=8).tolist() == [0, 8, 16]


def _optimal_radius(xyz, k):
    best = np.inf
    for sub in itertools.combinations(range(xyz.shape[0]), k):
        best = min(best, oa.covering_radius(xyz, np.asarray(sub)))
    return best


@pytest.mark.parametrize("seed", range(12))
def test_within_twice_the_optimal_covering_radius(seed):
    rng = np.random.default_rng(seed)
    xyz = rng.standard_normal((10, 3)) * rng.uniform(0.2, 3.0, size=3)
    for k in (2, 3, 4):
        got = oa.covering_radius(xyz, oa.farthest_point(xyz, k, start=seed % 10))
        assert got <= 2.0 * _optimal_radius(xyz, k) * (1 + 1e-12)


def test_output_invariants_and_shrinking_radius():
    rng = np.random.default_rng(5)
    xyz = rng.uniform(-1, 1, size=(300, 3))
    prev = np.inf
    for k in (1, 2, 5, 20, 80, 300):
        a = oa.farthest_point(xyz, k, start=17)
        assert a.dtype == np.int32 and a.shape == (k,)
        assert np.all(np.diff(a) > 0) and 17 in a
        r = oa.covering_radius(xyz, a)
        assert r <= prev
        prev = r
    assert prev == 0.0


def test_rejects_bad_arguments():
    xyz = _line(4)
    for n_c, start in ((0, 0), (5, 0), (2, 4), (2, -1)):
        with pytest.raises(ValueError):
            oa.farthest_point(xyz, n_c, start)
