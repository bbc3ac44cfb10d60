"""The rule the tile-level kernel uses, checked on CPU against the oracle's
definition (Sec. 4.2: a tile's level is the smallest level any of its pixels
needs).  A pixel's need is a non-decreasing function of its FP32 squared gaze
distance fl(fl(dx^2) + fl(dy^2)), which is non-decreasing in |dx| and |dy|, so
the minimum over a tile is reached at the pixel nearest the gaze; the kernel
evaluates the 4 x 4 pixels around it.  Here that rule is written in float32
numpy (each operation rounded, no fused multiply-add, as the kernel is built)
and compared with the oracle's per-pixel minimum on random rings, bands,
tile sizes and gazes inside, on and far outside the image."""
import numpy as np
import pytest

from paper_2407_00435_gb300 import synth

f32 = np.float32


def _need(gx, gy, R, L, band, x, y):
    dx = f32(f32(x) + f32(0.5)) - gx
    dy = f32(f32(y) + f32(0.5)) - gy
    d2 = f32(f32(dx * dx) + f32(dy * dy))
    lvl = 1
    for k in range(L - 1):
        if d2 >= f32(R[k] * R[k]):
            lvl += 1
    if lvl >= 2 and band > 0:
        Rb = f32(R[lvl - 2] + f32(band))
        if d2 < f32(Rb * Rb):
            return lvl - 1
    return lvl


def _rule_levels(W, H, tile, gx, gy, R, L, band):
    tx, ty = (W + tile - 1) // tile, (H + tile - 1) // tile
    out = np.zeros(tx * ty, np.uint8)
    for by in range(ty):
        for bx in range(tx):
            xa, xb = bx * tile, min(bx * tile + tile, W) - 1
            ya, yb = by * tile, min(by * tile + tile, H) - 1
            cx = int(np.floor(min(max(f32(gx - f32(0.5)), f32(xa - 2)), f32(xb + 2))))
            cy = int(np.floor(min(max(f32(gy - f32(0.5)), f32(ya - 2)), f32(yb + 2))))
            best = 255
            for lane in range(16):
                x = min(max(cx - 1 + (lane & 3), xa), xb)
                y = min(max(cy - 1 + (lane >> 2), ya), yb)
                best = min(best, _need(gx, gy, R, L, band, x, y))
            out[by * tx + bx] = best
    return out


@pytest.mark.parametrize("seed", range(4))
def test_nearest_pixel_rule_equals_per_pixel_minimum(orc, seed):
    rng = np.random.default_rng(100 + seed)
    levels_seen = set()
    for trial in range(12):
        W, H = int(rng.integers(20, 110)), int(rng.integers(20, 110))
        tile = int(rng.choice([8, 16]))
        L = int(rng.integers(2, 5))
        fy = f32(rng.uniform(30, 200))
        ring_tan = np.sort(rng.uniform(0.02, 1.2, L - 1)).astype(np.float32)
        band = float(rng.choice([0.0, 2.0, 7.5, 32.0]))
        kind = trial % 4
        if kind == 0:      # anywhere inside
            gx, gy = rng.uniform(0, W), rng.uniform(0, H)
        elif kind == 1:    # on a pixel centre
            gx, gy = rng.integers(0, W) + 0.5, rng.integers(0, H) + 0.5
        elif kind == 2:    # on a pixel corner
            gx, gy = float(rng.integers(0, W)), float(rng.integers(0, H))
        else:              # far outside
            gx, gy = rng.uniform(-3 * W, 4 * W), rng.uniform(-3 * H, 4 * H)
        gx, gy = f32(gx), f32(gy)
        row = synth.camera_lookat((0, 0, -5), (0, 0, 0), W, H)
        row[13] = fy
        cams = row.reshape(1, 20)
        fa = orc.FovArrays(L, np.zeros(1, np.uint8), ring_tan, band, np.array([gx, gy], np.float32))
        expect = orc.tile_levels(cams, tile, fa)
        R = (f32(cams[0, 13]) * ring_tan).astype(np.float32)
        got = _rule_levels(W, H, tile, gx, gy, R, L, band)
        np.testing.assert_array_equal(got, expect)
        levels_seen.update(int(v) for v in np.unique(expect))
    assert len(levels_seen) >= 2      # the cases reach more than one level
