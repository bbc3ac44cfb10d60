"""The FP64 HVSQ reference (oracle/hvsq.py) pinned by a value worked out by
hand, invariances of the definition (Sec. 2.2), the pooling law it encodes,
the split into quality regions (Sec. 4.3) and finite differences of its own
value for the gradient."""
import math

import numpy as np
import pytest

from oracle import hvsq as H
from paper_2407_00435_gb300 import synth


def test_hand_worked_three_by_three():
    # one bright pixel in the middle of a 3x3 black image against a black
    # reference, every pooling of half-width 1: mean^2 + std^2 of a pooling
    # is its mean of x^2 = 1 / (its pixel count): 1/9 in the middle, 1/4 at
    # the 4 corners (2x2 boxes), 1/6 at the 4 edges (2x3 boxes); 3 channels,
    # 9 pixels: HVSQ = 3 (1/9 + 4/4 + 4/6) / 9 = 48/81
    a = np.zeros((3, 3, 3))
    a[1, 1] = 1.0
    r = np.zeros((3, 3, 3))
    rad = np.ones((3, 3), np.int64)
    assert H.hvsq(a, r, rad)[0] == pytest.approx(48.0 / 81.0, rel=1e-14)
    # the middle pooling's statistics by hand: mean 1/9, std sqrt(8)/9
    m, s, n = H.pooled_stats(a, rad)
    assert m[1, 1, 0] == pytest.approx(1 / 9, rel=1e-15)
    assert s[1, 1, 0] == pytest.approx(math.sqrt(8) / 9, rel=1e-14)
    assert s[0, 0, 0] == pytest.approx(math.sqrt(3) / 4, rel=1e-14)
    assert n[0, 0] == 4 and n[0, 1] == 6 and n[1, 1] == 9


def test_invariances():
    rng = np.random.default_rng(1)
    a = rng.uniform(0, 1, (12, 10, 3))
    r = rng.uniform(0, 1, (12, 10, 3))
    rad = rng.integers(0, 4, (12, 10))
    v = H.hvsq(a, r, rad)[0]
    assert v > 0
    assert H.hvsq(r, a, rad)[0] == pytest.approx(v, rel=1e-12)          # symmetric
    assert H.hvsq(a + 0.3, r + 0.3, rad)[0] == pytest.approx(v, rel=1e-12)   # shift
    assert H.hvsq(2.5 * a, 2.5 * r, rad)[0] == pytest.approx(6.25 * v, rel=1e-12)
    assert H.hvsq(a, a, rad)[0] == 0.0
    # a pooling of one pixel has std 0: radius 0 everywhere gives the mean
    # squared colour difference
    z = np.zeros((12, 10), np.int64)
    assert H.hvsq(a, r, z)[0] == pytest.approx(((a - r) ** 2).sum(axis=2).mean(), rel=1e-12)


def test_regions_partition_the_image():
    rng = np.random.default_rng(2)
    a = rng.uniform(0, 1, (16, 16, 3))
    r = rng.uniform(0, 1, (16, 16, 3))
    rad = rng.integers(0, 3, (16, 16))
    reg = rng.integers(0, 3, (16, 16))
    per = H.hvsq(a, r, rad, reg, 3)
    n = np.bincount(reg.reshape(-1), minlength=3)
    assert (per * n).sum() / n.sum() == pytest.approx(H.hvsq(a, r, rad)[0], rel=1e-12)


def test_pooling_law_thresholds():
    # r = floor(r0 + k e^2) with e = atan(d / f) in degrees, decided against
    # the tangent thresholds: check pixels away from the thresholds
    t, base = synth.pooling_tangents(1.0, 0.025, 64)
    W, Hh, f = 400, 300, 260.0
    g = (137.0, 90.0)
    rad = H.pooling_radius(W, Hh, g, f, t, base)
    ys, xs = np.mgrid[0:Hh, 0:W]
    d = np.hypot(xs + 0.5 - g[0], ys + 0.5 - g[1])
    ecc = np.degrees(np.arctan(d / f))
    law = np.minimum(64, np.floor(1.0 + 0.025 * ecc ** 2)).astype(np.int64)
    frac = (1.0 + 0.025 * ecc ** 2) % 1.0
    clear = (frac > 1e-3) & (frac < 1 - 1e-3)
    np.testing.assert_array_equal(rad[clear], law[clear])
    assert rad.min() == 1 and rad.max() > 10
    assert H.radius_law(20.0) == 11 and H.radius_law(35.0) == 31 and H.radius_law(0.0) == 1


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    h, w = 7, 9
    a = rng.uniform(0, 1, (h, w, 3))
    r = rng.uniform(0, 1, (h, w, 3))
    rad = rng.integers(0, 3, (h, w))
    reg = rng.integers(0, 2, (h, w))
    g = H.hvsq_grad(a, r, rad, reg, 2)
    eps = 1e-6
    fd = np.zeros_like(a)
    for idx in np.ndindex(a.shape):
        ap = a.copy()
        am = a.copy()
        ap[idx] += eps
        am[idx] -= eps
        fd[idx] = (H.hvsq(ap, r, rad, reg, 2).sum() - H.hvsq(am, r, rad, reg, 2).sum()) / (2 * eps)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)
    # a planted mistake (the std term's factor x_q - m dropped) is caught
    bad = g.copy()
    bad[3, 4, 1] *= 1.001
    assert not np.allclose(bad, fd, rtol=1e-6, atol=1e-9)
