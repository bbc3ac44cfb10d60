"""Pins of the oracle's multi-model foveated render (Sec. 4.1, main pipeline:
each quality region rendered by a separate model, results blended in a band
outside each region boundary).  The foveated composite is checked against a
construction that shares none of its level logic: every level's model is
rendered on its own as a plain scene, and each pixel takes the image of its
level (and, inside a band, the linear mix with the level below), with the
pixel levels computed here in FP64 from the ring definition."""
import numpy as np
import pytest

from paper_2407_00435_gb300 import synth

RINGS_DEG = [7.0, 14.0]
BAND = 6.0
BG = (0.2, 0.1, 0.3)


def _setup(seed=31, n=1500, side=(128, 96)):
    rng = np.random.default_rng(seed)
    base = synth.uniform_scene(rng, n, degree=1, log_scale=(-3.0, 0.5), dc_mode="coef")
    cams = synth.camera_lookat((0.1, -0.05, -4), (0, 0, 0), side[0], side[1])[None]
    m = synth.nested_levels(rng, n, 3)
    sc, lv = synth.multi_model_scene(rng, base, m, 3)
    gaze = np.array([[0.45 * side[0], 0.55 * side[1]]], np.float32)
    fov = synth.Foveation(3, lv, synth.ring_tangents(RINGS_DEG), BAND, gaze, disjoint=True)
    return sc, lv, cams, fov


def _pixel_levels(cams, fov):
    """FP64 level, band flag, band weight and distance to the nearest decision
    boundary (relative, on squared distances) of every pixel of view 0."""
    W, H, fy = int(cams[0, 16]), int(cams[0, 17]), float(cams[0, 13])
    y, x = np.mgrid[0:H, 0:W]
    d2 = (x + 0.5 - float(fov.gaze[0, 0])) ** 2 + (y + 0.5 - float(fov.gaze[0, 1])) ** 2
    R = fy * np.asarray(fov.ring_tan, np.float64)
    lvl = 1 + (d2[..., None] >= R ** 2).sum(-1)
    d = np.sqrt(d2)
    Rprev = np.where(lvl >= 2, R[np.clip(lvl - 2, 0, len(R) - 1)], 0.0)
    band = (lvl >= 2) & (d < Rprev + fov.band_px)
    w = np.clip((d - Rprev) / fov.band_px, 0.0, 1.0)
    bounds = np.concatenate([R ** 2, (R + fov.band_px) ** 2])
    margin = np.min(np.abs(d2[..., None] - bounds) / bounds, axis=-1)
    return lvl.ravel(), band.ravel(), w.ravel(), margin.ravel()


def _sub(sc, sel):
    return synth.Scene(sc.means[sel], sc.scales[sel], sc.quats[sel], sc.opac[sel], sc.sh[sel],
                       sc.sh_degree)


def _per_level_images(orc, sc, lv, cams, tile, L):
    out = {}
    for level in range(1, L + 1):
        s = _sub(sc, np.nonzero(lv == level)[0])
        b = orc.bin_pairs(s, cams, tile)
        out[level] = orc.render(s, cams, tile, b, bg=BG).rgb
    return out


@pytest.mark.parametrize("tile", [16, 8])
def test_mmfr_equals_per_level_plain_renders(orc, tile):
    sc, lv, cams, fov = _setup()
    fa = orc.FovArrays.from_synth(fov)
    assert fa.disjoint
    bins = orc.bin_pairs(sc, cams, tile, fa)
    img = orc.render(sc, cams, tile, bins, fa, bg=BG)
    lvl, band, w, margin = _pixel_levels(cams, fov)
    assert set(np.unique(lvl)) == {1, 2, 3} and band.sum() > 50
    imgs = _per_level_images(orc, sc, lv, cams, tile, 3)
    exp = np.stack([imgs[l][i] for i, l in enumerate(lvl)])
    lower = np.stack([imgs[max(l - 1, 1)][i] for i, l in enumerate(lvl)])
    exp = np.where(band[:, None], w[:, None] * exp + (1.0 - w[:, None]) * lower, exp)
    ok = margin > 1e-5            # FP32 level decisions agree with FP64 there
    assert ok.mean() > 0.99
    np.testing.assert_allclose(img.rgb[ok], exp[ok], rtol=0, atol=1e-12)


def test_mmfr_tiled_equals_brute_force(orc):
    """Per-pixel lists of every visible point of the view (no tile filter,
    no tile ranges) give the same image: the tile filter keeps every point
    a pixel of the tile uses."""
    sc, lv, cams, fov = _setup(seed=5, n=600, side=(72, 56))
    fa = orc.FovArrays.from_synth(fov)
    bins = orc.bin_pairs(sc, cams, 8, fa)
    img = orc.render(sc, cams, 8, bins, fa, bg=BG)
    rgb, T, _ = orc.render_brute(sc, cams, 8, fa, bg=BG)
    np.testing.assert_allclose(img.rgb, rgb, rtol=0, atol=1e-12)
    np.testing.assert_allclose(img.T, T, rtol=0, atol=1e-12)


def test_mmfr_differs_from_nested(orc):
    """The same level tags read as nested quality bounds composite other
    points (finer models leak into coarser regions): the two modes must not
    coincide, or the membership rule would not be exercised."""
    sc, lv, cams, fov = _setup(seed=9, n=800)
    fa = orc.FovArrays.from_synth(fov)
    fn = orc.FovArrays.from_synth(fov)
    fn.disjoint = False
    a = orc.render(sc, cams, 16, orc.bin_pairs(sc, cams, 16, fa), fa, bg=BG).rgb
    b = orc.render(sc, cams, 16, orc.bin_pairs(sc, cams, 16, fn), fn, bg=BG).rgb
    lvl = _pixel_levels(cams, fov)[0]
    assert np.abs(a - b)[lvl == 1].max() > 1e-3
