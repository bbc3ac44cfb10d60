"""Pins of the pruning / scale-decay reference (Sec. 3.2-3.4) against hand
computations and brute force."""
import itertools

import numpy as np
import pytest

from oracle import prune as P


def test_ce_is_dominated_pixels_per_touched_tile_and_max_over_poses():
    # three points, two poses; point 2 is outside the first pose's view
    s1 = np.array([[4, 2, 0], [3, 1, 0], [40, 10, 0], [8, 1, 0]], np.uint32)
    s2 = np.array([[2, 5, 1], [2, 5, 1], [10, 50, 3], [1, 9, 2]], np.uint32)
    ce = P.ce_max([s1, s2])
    np.testing.assert_allclose(ce, [max(8 / 4, 1 / 2), max(1 / 2, 9 / 5), 2.0])
    assert P.ce_max([np.zeros((4, 3), np.uint32)]).tolist() == [0, 0, 0]


def test_prune_keep_is_the_lowest_ranks_by_ce_then_index():
    rng = np.random.default_rng(5)
    for n in (1, 7, 20):
        ce = rng.integers(0, 4, n).astype(np.float64) / 2     # many ties
        for fraction in (0.0, 0.1, 0.5, 0.99, 1.0):
            keep = P.prune_keep(ce, fraction)
            k = int(np.floor(fraction * n))
            assert (~keep).sum() == k
            # brute force: a point is removed iff fewer than k points come
            # before it in (ce, index) order
            for i in range(n):
                before = sum(1 for j in range(n) if (ce[j], j) < (ce[i], i))
                assert keep[i] == (before >= k)


def test_weighted_scale_by_hand_and_by_finite_differences():
    s = np.array([[1.0, 0.5, 0.2], [0.3, 2.0, 0.1], [0.2, 0.4, 3.0]])
    used = np.array([5, 10, 20])
    ws, g = P.weighted_scale(s, used, T=8)
    assert ws == pytest.approx((0 * 1.0 + 2 * 2.0 + 12 * 3.0) / 3)
    h = 1e-6
    for i, k in itertools.product(range(3), range(3)):
        sp, sm = s.copy(), s.copy()
        sp[i, k] += h
        sm[i, k] -= h
        fd = (P.weighted_scale(sp, used, 8)[0] - P.weighted_scale(sm, used, 8)[0]) / (2 * h)
        assert g[i, k] == pytest.approx(fd, abs=1e-6)
