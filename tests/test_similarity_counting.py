"""The counting identity the GPU's path-similarity kernel uses, checked on
the CPU against the oracle's definition (Sec. "Results": s(k, k') counts
the ordered contact pairs whose order relations agree in both paths).

With dense ranks x_i, y_i of the formation times of the two paths and the
joint histogram H[x][y], the number of agreeing ordered pairs is
    sum_cells c (c - 1) + 2 sum_cells c P,
c = H[x][y], P = number of contacts strictly below-left of the cell: pairs in
one cell tie in both paths, pairs of strictly ordered cells in the same
direction are concordant, every other pair disagrees.  Here the identity is
written out in numpy (not GPU code) and compared with the definition."""
import numpy as np
import pytest

import oracle as O


def _dense_ranks(t):
    v = np.where(t < 0, np.iinfo(np.int64).max, t)
    u = np.unique(v)
    return np.searchsorted(u, v), len(u)


def _agreements_from_histogram(ta, tb):
    x, ka = _dense_ranks(ta)
    y, kb = _dense_ranks(tb)
    H = np.zeros((ka, kb), np.int64)
    np.add.at(H, (x, y), 1)
    # P[x][y]: contacts with x' < x and y' < y
    P = np.zeros_like(H)
    P[1:, 1:] = np.cumsum(np.cumsum(H, axis=0), axis=1)[:-1, :-1]
    return int((H * (H - 1)).sum() + 2 * (H * P).sum())


@pytest.mark.parametrize("seed", range(6))
def test_histogram_count_equals_the_definition(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 300))
    hi = int(rng.choice([3, 20, 10 ** 6]))
    ta = rng.integers(-1, hi, n)
    tb = rng.integers(-1, hi, n) if seed % 2 else np.where(rng.random(n) < 0.3, -1, ta + rng.integers(0, 3, n))
    count = _agreements_from_histogram(ta, tb)
    assert count / (n * (n - 1)) == O.path_similarity(ta, tb)


def test_histogram_count_special_cases():
    t = np.arange(50)
    assert _agreements_from_histogram(t, t) == 50 * 49              # identical order: every pair agrees
    assert _agreements_from_histogram(t, 100 - t) == 0              # reversed: none
    u = -np.ones(50, np.int64)
    assert _agreements_from_histogram(u, u) == 50 * 49              # all ties in both
    assert _agreements_from_histogram(u, t) == 0                    # ties against a strict order
