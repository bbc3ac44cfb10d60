"""HVSQ, the eccentricity-aware visual quality metric, FP64 reference (TEST
INFRASTRUCTURE ONLY: only tests/ and the benchmark's CPU leg may import this
module).

Definition written out from the paper, Sec. 2.2 "Modeling HVS" (the HVSQ
equation) and Sec. 4.3 (HVSQ of one quality region as the quality loss):

  HVSQ = (1/N) sum_i [ (M(I^a_i) - M(I^r_i))^2 + (sigma(I^a_i) - sigma(I^r_i))^2 ]

over the N pixels i of an image (or of one region), I^a_i and I^r_i the
features of pixel i's spatial pooling in the altered and the reference image,
M the arithmetic mean and sigma the standard deviation.  The paper leaves the
feature model and the pooling law to an implementation it cites; readings:

* features: the three colour channels of the rendered image, each a feature;
  the squared differences are summed over the channels;
* pooling of pixel i: the square box of half-width r_i pixels around it,
  clipped to the image, r_i = floor(r0 + k e_i^2) with e_i the pixel's
  eccentricity in degrees (the angle between the gaze ray and the pixel's
  ray, atan(|p_i - g| / f): the geometry of the foveation rings); the paper
  says the pooling size grows with eccentricity, "usually quadratically".
  The integer r_i is decided as r_base + #{j : |p_i - g| >= f tan(theta_j)}
  with theta_j the eccentricities where r0 + k e^2 reaches r_base + 1,
  r_base + 2, ... (the caller's table of tangents, as for the rings), the
  distance compared squared in FP32 like the ring test, so the CUDA path and
  this reference take the same integer decisions.  Workload defaults r0 = 1,
  k = 0.025 per square degree (1 px at the fovea, 11 px at 20 deg, 31 px at
  35 deg), at most 64 px;
* sigma: the population standard deviation of the pooled values;
* the HVSQ of a region (Sec. 4.3) sums over the region's pixels and divides
  by their number; the loss of several regions is the sum of their HVSQs.

Gradient with respect to the altered image (the reference is fixed): for a
pooling i with n_i pixels, mean m_i and standard deviation s_i,
d m_i / d x_q = 1/n_i and d s_i / d x_q = (x_q - m_i) / (n_i s_i) for q in the
pooling (0 when s_i = 0: reading, the subgradient).
"""
from __future__ import annotations

import math

import numpy as np


def pooling_radius(width, height, gaze, focal, pool_tan, r_base=1):
    """(H, W) int array of the pooling half-widths: r_base plus the number of
    thresholds f tan(theta_j) the pixel's distance to the gaze reaches, the
    distance squared and compared in FP32 (dx = (x + 0.5) - gx, dx dx + dy dy,
    against (f t_j)^2)."""
    f32 = np.float32
    ys, xs = np.mgrid[0:height, 0:width]
    dx = (xs.astype(f32) + f32(0.5)) - f32(gaze[0])
    dy = (ys.astype(f32) + f32(0.5)) - f32(gaze[1])
    d2 = dx * dx + dy * dy
    r = np.full((height, width), int(r_base), np.int64)
    for t in np.asarray(pool_tan, f32):
        R = f32(focal) * t
        r += (d2 >= R * R).astype(np.int64)
    return r


def pooled_stats(img, radius):
    """Per pixel and channel: mean and population standard deviation of the
    image over the pixel's box (plain loops over pixels, numpy per box)."""
    H, W, C = img.shape
    mean = np.zeros((H, W, C))
    std = np.zeros((H, W, C))
    count = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            r = int(radius[y, x])
            box = img[max(0, y - r):min(H, y + r + 1), max(0, x - r):min(W, x + r + 1)]
            box = box.reshape(-1, C).astype(np.float64)
            m = box.mean(axis=0)
            mean[y, x] = m
            std[y, x] = np.sqrt(np.maximum(((box - m) ** 2).mean(axis=0), 0.0))
            count[y, x] = box.shape[0]
    return mean, std, count


def hvsq(alt, ref, radius, region=None, n_regions=1):
    """HVSQ per region (region: (H, W) ints in 0..n_regions-1, or None for
    one region, the whole image).  alt, ref: (H, W, 3)."""
    ma, sa, _ = pooled_stats(alt, radius)
    mr, sr, _ = pooled_stats(ref, radius)
    term = ((ma - mr) ** 2 + (sa - sr) ** 2).sum(axis=2)
    if region is None:
        region = np.zeros(term.shape, np.int64)
    out = np.zeros(n_regions)
    for g in range(n_regions):
        sel = region == g
        out[g] = term[sel].sum() / sel.sum() if sel.any() else 0.0
    return out


def hvsq_grad(alt, ref, radius, region=None, n_regions=1):
    """d (sum of the regions' HVSQs) / d alt, (H, W, 3): the chain rule of the
    definition above, pooling by pooling."""
    H, W, C = alt.shape
    ma, sa, cnt = pooled_stats(alt, radius)
    mr, sr, _ = pooled_stats(ref, radius)
    if region is None:
        region = np.zeros((H, W), np.int64)
    npx = np.bincount(region.reshape(-1), minlength=n_regions).astype(np.float64)
    g = np.zeros((H, W, C))
    a64 = alt.astype(np.float64)
    for y in range(H):
        for x in range(W):
            r = int(radius[y, x])
            y0, y1 = max(0, y - r), min(H, y + r + 1)
            x0, x1 = max(0, x - r), min(W, x + r + 1)
            w = 1.0 / npx[region[y, x]]
            n = cnt[y, x]
            dm = 2.0 * (ma[y, x] - mr[y, x]) * w
            ds = 2.0 * (sa[y, x] - sr[y, x]) * w
            box = a64[y0:y1, x0:x1]
            term = dm / n + np.where(sa[y, x] > 0,
                                     ds * (box - ma[y, x]) / (n * np.where(sa[y, x] > 0, sa[y, x], 1.0)),
                                     0.0)
            g[y0:y1, x0:x1] += term
    return g


def radius_law(ecc_deg, r0=1.0, k=0.025, r_max=64):
    """floor(r0 + k e^2), at most r_max (the law the thresholds encode)."""
    return min(int(r_max), int(math.floor(r0 + k * ecc_deg * ecc_deg)))
