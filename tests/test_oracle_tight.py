"""Pins of the oracle's opacity-aware tight support (a reading of the
paper's deferred support rule that shortens the tile lists without changing
the image).  A tile may be dropped only if no pixel centre in it can reach
alpha >= 1/255, which is checked here in FP64 from the value projection,
independently of the FP32 keyed test that makes the decision."""
import math

import numpy as np
import pytest

from paper_2407_00435_gb300 import synth

LOG_FLOOR = math.log(255.0)


def _views(rng, sizes):
    return synth.orbit_cameras(rng, len(sizes), 3.5, sizes)


def _scene(rng, n, degree=0):
    sc = synth.blob_scene(rng, n, n_blobs=6, degree=degree, log_scale=(-3.2, 0.6))
    # opacities across the whole range, some just above 1/255
    sc.opac[: n // 10] = rng.uniform(1.0 / 255.0, 0.02, n // 10).astype(np.float32)
    sc.opac[n // 10: n // 5] = rng.uniform(0.95, 0.999, n // 10).astype(np.float32)
    return sc


def _dropped_tiles_never_blend(orc, sc, cams, tile, fov=None, o_max=None):
    b_rect = orc.bin_pairs(sc, cams, tile, fov)
    b_tight = orc.bin_pairs(sc, cams, tile, fov, tight=True)
    vp = orc.project_values(sc, cams, b_rect.vis)
    n = sc.n
    o = sc.opac.astype(np.float64) if o_max is None else o_max
    W, H, tx, ty = orc.view_dims(cams, tile)
    checked = dropped = 0
    for it in np.nonzero(b_rect.vis == 1)[0]:
        v, i = divmod(int(it), n)
        x0, x1, y0, y1 = b_rect.rect[it]
        u, vv = vp[it, orc.ORC_U], vp[it, orc.ORC_V]
        A, B, Cc = vp[it, orc.ORC_CA], vp[it, orc.ORC_CB], vp[it, orc.ORC_CC]
        tau = 2.0 * (LOG_FLOOR + math.log(o[i])) if o[i] > 0 else -1.0
        keep = set()
        tb = int((tx[:v] * ty[:v]).sum())
        for y in range(y0, y1 + 1):
            for x in range(x0, x1 + 1):
                t = tb + y * tx[v] + x
                s, e = b_tight.ranges[t]
                if np.any(b_tight.vals[s:e] == v * n + i):
                    keep.add((x, y))
        for y in range(y0, y1 + 1):
            for x in range(x0, x1 + 1):
                t = tb + y * tx[v] + x
                if b_rect.tile_level is not None and fov is not None:
                    if b_rect.tile_level[t] > fov.bound_m[i]:
                        continue
                checked += 1
                if (x, y) in keep:
                    continue
                dropped += 1
                px = np.arange(x * tile, min((x + 1) * tile, W[v])) + 0.5 - u
                py = np.arange(y * tile, min((y + 1) * tile, H[v])) + 0.5 - vv
                dx, dy = np.meshgrid(px, py)
                q = A * dx * dx + 2 * B * dx * dy + Cc * dy * dy
                assert q.min() > tau, (it, x, y, q.min(), tau)
    return checked, dropped, b_rect, b_tight


def test_tight_support_drops_only_tiles_that_cannot_blend(orc):
    rng = np.random.default_rng(31)
    sc = _scene(rng, 1500, degree=1)
    cams = _views(rng, [(96, 80), (72, 100)])
    checked, dropped, b_rect, b_tight = _dropped_tiles_never_blend(orc, sc, cams, 16)
    assert dropped > 0.3 * checked           # the test is not vacuous
    assert b_tight.K == int(b_tight.counts.sum()) < b_rect.K


def test_tight_support_covers_the_largest_level_opacity(orc):
    rng = np.random.default_rng(32)
    sc = _scene(rng, 1200)
    cams = _views(rng, [(80, 80)])
    m = synth.nested_levels(rng, sc.n, 3)
    f = synth.Foveation(3, m, synth.ring_tangents([6, 12]), 6.0, synth.random_gaze(rng, cams))
    op_lv, dc_lv = synth.multiversion_params(rng, sc, 3)
    op_lv = np.ascontiguousarray(op_lv, np.float32)
    op_lv[:, : sc.n // 3] = 0.99          # level opacities far above the base one
    fa = orc.FovArrays.from_synth(f, op_lv, dc_lv)
    o_max = np.maximum(sc.opac.astype(np.float64), op_lv.astype(np.float64).max(axis=0))
    checked, dropped, _, _ = _dropped_tiles_never_blend(orc, sc, cams, 16, fa, o_max)
    assert dropped > 0.2 * checked


def test_tight_support_keeps_the_image(orc):
    rng = np.random.default_rng(33)
    sc = _scene(rng, 2500, degree=2)
    cams = _views(rng, [(112, 96), (64, 64)])
    b_rect = orc.bin_pairs(sc, cams, 16)
    b_tight = orc.bin_pairs(sc, cams, 16, tight=True)
    assert b_tight.K < 0.8 * b_rect.K
    i_rect = orc.render(sc, cams, 16, b_rect)
    i_tight = orc.render(sc, cams, 16, b_tight)
    np.testing.assert_allclose(i_tight.rgb, i_rect.rgb, rtol=0, atol=1e-12)
    np.testing.assert_allclose(i_tight.T, i_rect.T, rtol=0, atol=1e-12)
    # the last blended point is the same point (its list position differs)
    W, H, tx, ty = orc.view_dims(cams, 16)
    pix = np.arange(len(i_rect.rgb))
    base = np.concatenate([[0], np.cumsum(W * H)])
    tbase = np.concatenate([[0], np.cumsum(tx * ty)])
    for p in pix[::7]:
        v = int(np.searchsorted(base, p, side="right") - 1)
        y, x = divmod(int(p - base[v]), int(W[v]))
        t = tbase[v] + (y // 16) * tx[v] + x // 16
        lr, lt = i_rect.last[p, 0], i_tight.last[p, 0]
        assert (lr < 0) == (lt < 0)
        if lr >= 0:
            assert b_rect.vals[b_rect.ranges[t, 0] + lr] == b_tight.vals[b_tight.ranges[t, 0] + lt]


def test_tight_support_disc_closed_form(orc):
    # one isotropic point on the axis: Sigma' = (f s / z)^2 I + 0.3 I, so
    # the support is a disc of radius sqrt(tau) sigma' around the mean
    f, z, s, o = 100.0, 5.0, 0.4, 0.8
    cam = np.zeros(20, np.float32)
    cam[[0, 4, 8]] = 1.0
    cam[12:20] = [f, f, 128.0, 96.0, 256, 192, 0.2, 100.0]
    sc = synth.Scene(np.array([[0.13, -0.07, z]], np.float32), np.full((1, 3), s, np.float32),
                     np.array([[1.0, 0, 0, 0]], np.float32), np.array([o], np.float32),
                     np.zeros((1, 1, 3), np.float32), 0)
    b = orc.bin_pairs(sc, cam[None], 16, tight=True)
    b_rect = orc.bin_pairs(sc, cam[None], 16)
    sig2 = (f * s / z) ** 2 + 0.3
    u, v = f * 0.13 / z + 128.0, f * -0.07 / z + 96.0
    r_true = math.sqrt(2 * (LOG_FLOOR + math.log(o)) * sig2)
    # the bound ln x <= e ln2 + (m - 1) overshoots by at most 1 - ln 2
    r_up = math.sqrt((2 * (LOG_FLOOR + math.log(o) + 1 - math.log(2)) * (1 + 2 ** -10) + 2 ** -10) * sig2)
    x0, x1, y0, y1 = b_rect.rect[0]
    for y in range(y0, y1 + 1):
        for x in range(x0, x1 + 1):
            # nearest point of the tile's pixel-centre rectangle to the mean
            cx = min(max(u, x * 16 + 0.5), x * 16 + 15.5)
            cy = min(max(v, y * 16 + 0.5), y * 16 + 15.5)
            d = math.hypot(cx - u, cy - v)
            s_, e_ = b.ranges[y * 16 + x]
            kept = e_ > s_
            if d <= r_true * (1 - 1e-6):
                assert kept, (x, y, d, r_true)
            if d > r_up * (1 + 1e-6):
                assert not kept, (x, y, d, r_up)


def test_tight_support_without_any_blendable_pixel(orc):
    # opacity below 1/255: no pixel can blend, so no pair survives
    rng = np.random.default_rng(34)
    sc = _scene(rng, 300)
    sc.opac[:] = 0.5 / 255.0
    b = orc.bin_pairs(sc, _views(rng, [(64, 64)]), 16, tight=True)
    assert (b.vis == 1).sum() > 100 and b.K == 0


@pytest.mark.parametrize("band", [0.0, 6.0, 40.0])
def test_tile_levels_at_most_m_are_one_interval_per_row(orc, band):
    # the foveation filter keeps a pair iff tile level <= m; per tile row those
    # tiles form one run of columns (levels first fall, then rise along a row)
    rng = np.random.default_rng(35)
    for trial in range(6):
        W, H = int(rng.integers(40, 300)), int(rng.integers(40, 300))
        cams = synth.orbit_cameras(rng, 1, 3.0, [(W, H)])
        L = int(rng.integers(2, 6))
        rings = np.sort(rng.uniform(3, 40, L - 1))
        gaze = np.array([[rng.uniform(-0.2, 1.2) * W, rng.uniform(-0.2, 1.2) * H]], np.float32)
        f = synth.Foveation(L, np.ones(10, np.uint8), synth.ring_tangents(list(rings)), band, gaze)
        for tile in (16, 8):
            tl = orc.tile_levels(cams, tile, orc.FovArrays.from_synth(f))
            tx, ty = (W + tile - 1) // tile, (H + tile - 1) // tile
            lv = tl.reshape(ty, tx)
            for m in range(1, L + 1):
                for row in lv:
                    cols = np.nonzero(row <= m)[0]
                    if len(cols):
                        assert cols[-1] - cols[0] + 1 == len(cols), (trial, tile, m, row)
