"""Pins of the FP64 oracle against things other than itself.

Each test fixes part of the oracle with an independent source: a closed form
worked out by hand, SciPy's spherical harmonics and rotations, a numerical
Jacobian of the pinhole map, brute-force per-pixel compositing, numpy's
stable sort, invariants of Eq. 1, or finite differences of the oracle's own
forward pass.  None of them re-types the oracle's formula.
"""
import math

import numpy as np
import pytest

from paper_2407_00435_gb300 import synth

Y00 = 0.5 / math.sqrt(math.pi)


def axis_camera(W, H, f, znear=0.2, zfar=1000.0):
    """Camera at the origin looking down +z (R = I, t = 0)."""
    row = np.zeros(20, np.float32)
    row[[0, 4, 8]] = 1.0
    row[12:20] = [f, f, W / 2, H / 2, W, H, znear, zfar]
    return row[None]


def make_scene(means, scales, quats=None, opac=None, sh=None, degree=0):
    n = len(means)
    if quats is None:
        quats = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    if opac is None:
        opac = np.full(n, 0.5)
    if sh is None:
        sh = np.zeros((n, (degree + 1) ** 2, 3))
    return synth.Scene(np.asarray(means, np.float32), np.asarray(scales, np.float32),
                       np.asarray(quats, np.float32), np.asarray(opac, np.float32),
                       np.asarray(sh, np.float32), degree)


def dc_for_rgb(rgb):
    return (np.asarray(rgb, np.float64) - 0.5) / Y00


# ---------------------------------------------------------------------------
# g (Eq. 1c): real spherical harmonics against SciPy
# ---------------------------------------------------------------------------
def test_sh_basis_matches_scipy(orc):
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(0)
    for _ in range(50):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        theta = math.acos(max(-1.0, min(1.0, d[2])))
        phi = math.atan2(d[1], d[0]) % (2 * math.pi)
        Y = orc.sh_basis(d)
        for l in range(4):
            for m in range(-l, l + 1):
                if m == 0:
                    ref = sph_harm_y(l, 0, theta, phi).real
                elif m > 0:
                    ref = math.sqrt(2) * sph_harm_y(l, m, theta, phi).real
                else:
                    ref = math.sqrt(2) * sph_harm_y(l, -m, theta, phi).imag
                assert abs(Y[l * l + l + m] - ref) < 1e-12, (l, m)


def test_sh_colour_degree0_and_view_dependence(orc):
    # degree 0: colour = Y00 * dc + 0.5, clamped at zero
    cams = axis_camera(32, 32, 60.0)
    sc = make_scene([[0, 0, 4], [0.1, 0, 4]], [[0.05] * 3] * 2,
                    sh=[[[0.3, -0.2, -5.0]], [[1.0, 0.0, 0.5]]])
    vis, _, _ = orc.keyed_project(sc, cams, 16)
    vp = orc.project_values(sc, cams, vis)
    exp0 = np.maximum(0, Y00 * np.array([0.3, -0.2, -5.0]) + 0.5)
    np.testing.assert_allclose(vp[0, orc.ORC_R:orc.ORC_B + 1], exp0, atol=1e-7)
    # degree 1: a coefficient on the z-harmonic tracks the view direction
    sh = np.zeros((1, 4, 3))
    sh[0, 2, :] = 1.0  # Y_1^0 ~ z
    sc1 = make_scene([[0.0, 0.0, 4.0]], [[0.05] * 3], sh=sh, degree=1)
    vis, _, _ = orc.keyed_project(sc1, cams, 16)
    vp = orc.project_values(sc1, cams, vis)
    # direction from the camera (origin) to the mean is +z
    np.testing.assert_allclose(vp[0, orc.ORC_R], 0.5 + math.sqrt(3 / (4 * math.pi)), atol=1e-7)


# ---------------------------------------------------------------------------
# f (Eq. 1b) and the EWA splat: closed forms
# ---------------------------------------------------------------------------
def test_single_isotropic_gaussian_closed_form(orc):
    W = H = 32
    f, z, sig, o = 100.0, 4.0, 0.05, 0.8
    cams = axis_camera(W, H, f)
    rgb = np.array([0.9, 0.4, 0.1])
    sc = make_scene([[0, 0, z]], [[sig] * 3], opac=[o], sh=[[dc_for_rgb(rgb)]])
    bins = orc.bin_pairs(sc, cams, 16)
    img = orc.render(sc, cams, 16, bins)
    s2 = (f * float(np.float32(sig)) / z) ** 2 + 0.3   # Sigma' = (f sigma / z)^2 I + 0.3 I
    ys, xs = np.mgrid[0:H, 0:W]
    d2 = (xs + 0.5 - W / 2) ** 2 + (ys + 0.5 - H / 2) ** 2
    alpha = np.minimum(0.99, float(np.float32(o)) * np.exp(-0.5 * d2 / s2))
    alpha = np.where(alpha < 1 / 255, 0.0, alpha)
    col = dc_for_rgb(rgb).astype(np.float32).astype(np.float64) * Y00 + 0.5
    expect = alpha[..., None] * col[None, None, :]
    np.testing.assert_allclose(img.rgb.reshape(H, W, 3), expect, atol=1e-6, rtol=1e-6)
    np.testing.assert_allclose(img.T[:, 0].reshape(H, W), 1 - alpha, atol=1e-6)


def _rotation_scipy(q_wxyz):
    from scipy.spatial.transform import Rotation
    w, x, y, z = q_wxyz
    return Rotation.from_quat([x, y, z, w]).as_matrix()


def _num_jacobian(p, fx, fy, cx, cy):
    def proj(q):
        return np.array([fx * q[0] / q[2] + cx, fy * q[1] / q[2] + cy])
    J = np.zeros((2, 3))
    for k in range(3):
        h = 1e-6 * max(1.0, abs(p[k]))
        e = np.zeros(3)
        e[k] = h
        J[:, k] = (proj(p + e) - proj(p - e)) / (2 * h)
    return J


def test_2d_covariance_against_scipy_rotation_and_numerical_jacobian(orc):
    rng = np.random.default_rng(3)
    cam = synth.camera_lookat((0.3, -0.5, -4.0), (0, 0, 0), 200, 150)
    sc = synth.uniform_scene(rng, 40, degree=0, log_scale=(-3.0, 0.6))
    vis, _, _ = orc.keyed_project(sc, cam[None], 16)
    vp = orc.project_values(sc, cam[None], vis)
    R = cam[:9].astype(np.float64).reshape(3, 3)
    t = cam[9:12].astype(np.float64)
    fx, fy, cx, cy = cam[12:16].astype(np.float64)
    checked = 0
    for i in np.nonzero(vis == 1)[0]:
        mu = sc.means[i].astype(np.float64)
        p = R @ mu + t
        if abs(p[0] / p[2]) > 1.3 * 0.5 * 200 / fx or abs(p[1] / p[2]) > 1.3 * 0.5 * 150 / fy:
            continue  # J's clamp active: not the plain pinhole Jacobian
        Rq = _rotation_scipy(sc.quats[i].astype(np.float64))
        Sig = Rq @ np.diag(sc.scales[i].astype(np.float64) ** 2) @ Rq.T
        J = _num_jacobian(p, fx, fy, cx, cy)
        S2 = J @ R @ Sig @ R.T @ J.T + 0.3 * np.eye(2)
        got = vp[i, [orc.ORC_SA, orc.ORC_SB, orc.ORC_SC]]
        np.testing.assert_allclose(got, [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-7,
                                   atol=1e-9 * S2[0, 0])
        conic = np.linalg.inv(S2)
        np.testing.assert_allclose(vp[i, [orc.ORC_CA, orc.ORC_CB, orc.ORC_CC]],
                                   [conic[0, 0], conic[0, 1], conic[1, 1]], rtol=1e-6)
        # 2D mean = pinhole projection of the 3D mean
        np.testing.assert_allclose(vp[i, [orc.ORC_U, orc.ORC_V]],
                                   [fx * p[0] / p[2] + cx, fy * p[1] / p[2] + cy], rtol=1e-12)
        checked += 1
    assert checked > 20


def _clamped_cov(p, Sig, fx, fy, cx, cy, limx, limy, how="right"):
    """Sigma' = J Sigma J^T + 0.3 I with J the numerical Jacobian of the
    pinhole map at the camera-space point whose x/z, y/z are clamped to
    +-lim (camera rotation = identity).  `how` plants the mistakes the pin
    must tell apart."""
    tx, ty = p[0] / p[2], p[1] / p[2]
    if how == "swap":            # the width's limit used for y and vice versa
        limx, limy = limy, limx
    if how == "sign":            # clamped to the wrong side
        cxl = -np.clip(tx, -limx, limx) if abs(tx) > limx else tx
        cyl = -np.clip(ty, -limy, limy) if abs(ty) > limy else ty
    elif how == "none":
        cxl, cyl = tx, ty
    else:
        cxl, cyl = np.clip(tx, -limx, limx), np.clip(ty, -limy, limy)
    q = np.array([cxl * p[2], cyl * p[2], p[2]])
    J = _num_jacobian(q, fx, fy, cx, cy)
    return J @ Sig @ J.T + 0.3 * np.eye(2)


def test_jacobian_clamp_outside_the_frustum(orc):
    # Reading: J of the EWA splat is evaluated at the camera-space mean with
    # x/z and y/z clamped to 1.3 tan(half field of view) of each axis
    # (horizontal: (W/2)/fx, vertical: (H/2)/fy); the 2D mean is not
    # clamped.  Points beyond the clamp on every side, the image wider than
    # tall so that the two limits differ (1.3 vs 0.78).
    W, H, f = 200, 120, 100.0
    cam = axis_camera(W, H, f)
    limx, limy = 1.3 * (W / 2) / f, 1.3 * (H / 2) / f
    z = 2.0
    ratios = [(1.6, 0.0), (-1.6, 0.2), (0.2, 1.0), (0.1, -1.0), (1.5, -0.9), (-1.5, 0.9),
              (0.5, 0.3), (-1.45, -0.5)]
    means = np.array([[a * z, b * z, z] for a, b in ratios])
    rng = np.random.default_rng(17)
    scales = np.exp(rng.normal(np.log(0.5), 0.3, (len(means), 3)))
    quats = rng.normal(size=(len(means), 4))
    sc = make_scene(means, scales, quats=quats)
    vis, _, _, supp = orc.keyed_project(sc, cam, 16, tight=True)
    assert np.all(vis == 1), vis
    vp = orc.project_values(sc, cam, vis)
    n_clamped = 0
    mistakes = {"swap": 0.0, "sign": 0.0, "none": 0.0}
    for i, (a, b) in enumerate(ratios):
        p = sc.means[i].astype(np.float64)
        Rq = _rotation_scipy(sc.quats[i].astype(np.float64) / np.linalg.norm(sc.quats[i]))
        Sig = Rq @ np.diag(sc.scales[i].astype(np.float64) ** 2) @ Rq.T
        S2 = _clamped_cov(p, Sig, f, f, W / 2, H / 2, limx, limy)
        got = vp[i, [orc.ORC_SA, orc.ORC_SB, orc.ORC_SC]]
        want = [S2[0, 0], S2[0, 1], S2[1, 1]]
        np.testing.assert_allclose(got, want, rtol=1e-7, atol=1e-9 * S2[0, 0])
        # the keyed FP32 covariance (binning) takes the same clamp
        np.testing.assert_allclose(supp[i, 2:5], want, rtol=2e-5, atol=2e-6 * S2[0, 0])
        # 2D mean: the unclamped pinhole projection
        np.testing.assert_allclose(vp[i, [orc.ORC_U, orc.ORC_V]],
                                   [f * p[0] / p[2] + W / 2, f * p[1] / p[2] + H / 2], rtol=1e-12)
        n_clamped += abs(a) > limx or abs(b) > limy
        for how in mistakes:
            M = _clamped_cov(p, Sig, f, f, W / 2, H / 2, limx, limy, how)
            d = np.abs(np.array([M[0, 0], M[0, 1], M[1, 1]]) - want).max() / S2[0, 0]
            mistakes[how] = max(mistakes[how], d)
    assert n_clamped >= 6
    # each planted mistake moves some covariance far beyond the tolerance
    assert all(v > 1e-3 for v in mistakes.values()), mistakes


def test_keyed_rect_covers_three_sigma_and_depth_is_camera_z(orc):
    # The tile rectangle is the set of tiles overlapped by the square of
    # half-width ceil(3 sqrt(lambda_max)) around the 2D mean: it must contain
    # the tiles of the exact 3-sigma square and none beyond 3 sigma + 1 px
    # (sigma taken with the eigenvalue-gap floor of the radius reading).
    rng = np.random.default_rng(5)
    W, H, B = 160, 96, 16
    cam = synth.camera_lookat((0.0, 0.0, -4.0), (0, 0, 0), W, H)
    sc = synth.uniform_scene(rng, 300, degree=0, log_scale=(-3.0, 0.6))
    vis, dbits, rect = orc.keyed_project(sc, cam[None], B)
    vp = orc.project_values(sc, cam[None], vis)
    tx, ty = W // B, H // B
    n_ok = 0
    for i in np.nonzero(vis == 1)[0]:
        S2 = np.array([[vp[i, orc.ORC_SA], vp[i, orc.ORC_SB]],
                       [vp[i, orc.ORC_SB], vp[i, orc.ORC_SC]]])
        lam = np.linalg.eigvalsh(S2).max()
        r = 3 * math.sqrt(lam)
        # the radius reading floors the eigenvalue gap at sqrt(0.1)
        r_hi = 3 * math.sqrt(max(lam, 0.5 * np.trace(S2) + math.sqrt(0.1))) + 1
        u, v = vp[i, orc.ORC_U], vp[i, orc.ORC_V]
        x0, x1, y0, y1 = rect[i]
        e = 1e-3
        assert x0 <= max(0, math.floor((u - r + e) / B)) and x0 >= max(0, math.floor((u - r_hi - e) / B))
        assert x1 >= min(tx - 1, math.floor((u + r - e) / B)) and x1 <= min(tx - 1, math.floor((u + r_hi + e) / B))
        assert y0 <= max(0, math.floor((v - r + e) / B)) and y0 >= max(0, math.floor((v - r_hi - e) / B))
        assert y1 >= min(ty - 1, math.floor((v + r - e) / B)) and y1 <= min(ty - 1, math.floor((v + r_hi + e) / B))
        z = np.frombuffer(np.uint32(dbits[i]).tobytes(), np.float32)[0]
        assert abs(float(z) - vp[i, orc.ORC_DEPTH]) <= 4 * float(np.spacing(np.float32(z)))
        n_ok += 1
    assert n_ok > 100


# ---------------------------------------------------------------------------
# Eq. 1a: compositing worked out by hand
# ---------------------------------------------------------------------------
def _alpha_iso(o, f, sig, z, d2):
    s2 = (f * float(np.float32(sig)) / z) ** 2 + 0.3
    return min(0.99, float(np.float32(o)) * math.exp(-0.5 * d2 / s2))


def test_two_gaussians_by_hand(orc):
    W = H = 32
    f = 80.0
    c1, c2 = np.array([1.0, 0.2, 0.1]), np.array([0.1, 0.3, 0.9])
    sc = make_scene([[0, 0, 2.0], [0, 0, 3.0]], [[0.04] * 3, [0.09] * 3], opac=[0.6, 0.7],
                    sh=[[dc_for_rgb(c1)], [dc_for_rgb(c2)]])
    cams = axis_camera(W, H, f)
    bins = orc.bin_pairs(sc, cams, 16)
    px = np.array([16 * W + 16, 18 * W + 13])  # pixels (16,16) and (13,18)
    img = orc.render(sc, cams, 16, bins, pix=px)
    for q, (x, y) in enumerate([(16, 16), (13, 18)]):
        d2 = (x + 0.5 - 16) ** 2 + (y + 0.5 - 16) ** 2
        a1 = _alpha_iso(0.6, f, 0.04, 2.0, d2)
        a2 = _alpha_iso(0.7, f, 0.09, 3.0, d2)
        a1 = 0 if a1 < 1 / 255 else a1
        a2 = 0 if a2 < 1 / 255 else a2
        col1 = dc_for_rgb(c1).astype(np.float32).astype(np.float64) * Y00 + 0.5
        col2 = dc_for_rgb(c2).astype(np.float32).astype(np.float64) * Y00 + 0.5
        expect = a1 * col1 + (1 - a1) * a2 * col2
        np.testing.assert_allclose(img.rgb[q], expect, atol=1e-7)
        np.testing.assert_allclose(img.T[q, 0], (1 - a1) * (1 - a2), atol=1e-7)


def test_early_stop_excludes_the_stopping_point_and_clamp(orc):
    # four nearly opaque splats stacked on the axis; at the centre pixel each
    # has alpha = 0.95, so T = 0.05, 0.0025, 1.25e-4 and the fourth would take
    # T to 6.25e-6 < 1e-4: it is not blended (stop before adding it).
    W = H = 16
    f = 50.0
    z = np.array([2.0, 2.5, 3.0, 3.5])
    sig = 0.5 * z / f                       # footprint of 0.5 px std at every depth
    s2 = (f * sig.astype(np.float32).astype(np.float64) / z) ** 2 + 0.3
    d2 = 0.5  # pixel (8, 8) centre is (8.5, 8.5), mean at (8, 8)
    o = 0.95 / np.exp(-0.5 * d2 / s2)
    cols = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], np.float64) * 0.8 + 0.1
    sc = make_scene(np.stack([np.zeros(4), np.zeros(4), z], 1), np.repeat(sig[:, None], 3, 1),
                    opac=o, sh=dc_for_rgb(cols)[:, None, :])
    cams = axis_camera(W, H, f)
    bins = orc.bin_pairs(sc, cams, 16)
    img = orc.render(sc, cams, 16, bins, pix=np.array([8 * W + 8]))
    a = o.astype(np.float32).astype(np.float64) * np.exp(-0.5 * d2 / s2)
    col = dc_for_rgb(cols).astype(np.float32).astype(np.float64) * Y00 + 0.5
    T = 1.0
    expect = np.zeros(3)
    for k in range(3):
        expect += T * a[k] * col[k]
        T *= 1 - a[k]
    assert T * (1 - a[3]) < 1e-4
    np.testing.assert_allclose(img.rgb[0], expect, atol=1e-9)
    np.testing.assert_allclose(img.T[0, 0], T, rtol=1e-9)
    assert img.last[0, 0] == 2
    # clamp: an opacity above 0.99 at the peak is clamped to 0.99
    sig2 = 20.0 * 2.0 / f                   # 20 px footprint: nearly flat peak
    sc2 = make_scene([[0, 0, 2.0]], [[sig2] * 3], opac=[0.9999], sh=[[dc_for_rgb([1, 1, 1])]])
    img2 = orc.render(sc2, cams, 16, orc.bin_pairs(sc2, cams, 16), pix=np.array([8 * W + 8]))
    s22 = (f * float(np.float32(sig2)) / 2.0) ** 2 + 0.3
    a0 = float(np.float32(0.9999)) * math.exp(-0.5 * d2 / s22)
    assert a0 > 0.99
    np.testing.assert_allclose(img2.T[0, 0], 0.01, rtol=1e-12)


# ---------------------------------------------------------------------------
# binning, sorting, ranges: brute force and numpy's stable sort
# ---------------------------------------------------------------------------
def _emitted(orc, sc, cams, tile, fov=None):
    vis, dbits, rect = orc.keyed_project(sc, cams, tile)
    n, V = sc.n, len(cams)
    W, H, tx, ty = orc.view_dims(cams, tile)
    tbase = np.concatenate([[0], np.cumsum(tx * ty)])
    tl = orc.tile_levels(cams, tile, fov) if fov is not None else None
    keys, vals = [], []
    for v in range(V):
        for i in range(n):
            it = v * n + i
            if vis[it] != 1:
                continue
            x0, x1, y0, y1 = rect[it]
            for y in range(y0, y1 + 1):
                for x in range(x0, x1 + 1):
                    gt = tbase[v] + y * tx[v] + x
                    if tl is not None and tl[gt] > fov.bound_m[i]:
                        continue
                    keys.append((int(gt) << 32) | int(dbits[it]))
                    vals.append(it)
    return np.array(keys, np.uint64), np.array(vals, np.uint32), tbase[-1]


def _small_fov(rng, n, V, cams, levels=4, band=6.0, mv=False, sc=None):
    m = synth.nested_levels(rng, n, levels)
    gaze = synth.random_gaze(rng, cams)
    f = synth.Foveation(levels, m, synth.ring_tangents([5, 10, 18][:levels - 1]), band, gaze)
    op = dc = None
    if mv:
        op, dc = synth.multiversion_params(rng, sc, levels)
    return f, op, dc


def test_sort_and_ranges_match_numpy_stable_sort(orc):
    rng = np.random.default_rng(11)
    sc = synth.uniform_scene(rng, 400, degree=0, log_scale=(-3.2, 0.6))
    cams = synth.orbit_cameras(rng, 3, 4.0, [(64, 48), (40, 72), (96, 96)])
    for fov in (None, "fov"):
        fa = None
        if fov:
            f, _, _ = _small_fov(rng, sc.n, 3, cams)
            fa = orc.FovArrays.from_synth(f)
        keys, vals, T = _emitted(orc, sc, cams, 16, fa)
        order = np.argsort(keys, kind="stable")
        b = orc.bin_pairs(sc, cams, 16, fa)
        np.testing.assert_array_equal(b.keys, keys[order])
        np.testing.assert_array_equal(b.vals, vals[order])
        tiles = (keys[order] >> np.uint64(32)).astype(np.int64)
        for t in range(T):
            idx = np.nonzero(tiles == t)[0]
            if len(idx):
                assert tuple(b.ranges[t]) == (idx[0], idx[-1] + 1)
            else:
                assert b.ranges[t, 0] == b.ranges[t, 1]
        assert int(b.counts.sum()) == len(keys)


@pytest.mark.parametrize("fov_mode", [None, "fov", "fov_mv"])
def test_tiled_equals_brute_force(orc, fov_mode):
    rng = np.random.default_rng(21)
    sc = synth.uniform_scene(rng, 64, degree=3, log_scale=(-2.8, 0.5), dc_mode="coef")
    cams = synth.orbit_cameras(rng, 2, 3.0, [(32, 32), (48, 40)])
    fa = None
    if fov_mode:
        f, op, dc = _small_fov(rng, sc.n, 2, cams, mv=(fov_mode == "fov_mv"), sc=sc)
        fa = orc.FovArrays.from_synth(f, op, dc)
    b = orc.bin_pairs(sc, cams, 16, fa)
    img = orc.render(sc, cams, 16, b, fa)
    # the brute force applies no tile filter: for foveated views the tiled
    # result equals it only if the tile levels are conservative (Sec. 4.2)
    rgb, T, last_item = orc.render_brute(sc, cams, 16, fa)
    np.testing.assert_array_equal(img.rgb, rgb)
    np.testing.assert_array_equal(img.T, T)
    np.testing.assert_array_equal(_last_items(orc, b, cams, 16, img.last), last_item)
    assert (img.last[:, 0] >= 0).mean() > 0.1
    if fa is not None:
        # the filter does drop pairs here, so the comparison exercises it
        b0 = orc.bin_pairs(sc, cams, 16)
        assert b.K < b0.K


def _last_items(orc, b, cams, tile, last):
    """Tile-list positions of `last` (P, 2) -> items (v*N + i), -1 kept."""
    W, H, tx, ty = orc.view_dims(cams, tile)
    tbase = np.concatenate([[0], np.cumsum(tx * ty)])
    out = np.full(last.shape, -1, np.int64)
    q = 0
    for v in range(len(cams)):
        ys, xs = np.divmod(np.arange(W[v] * H[v]), W[v])
        gt = tbase[v] + (ys // tile) * tx[v] + xs // tile
        for a in range(2):
            lv = last[q:q + W[v] * H[v], a].astype(np.int64)
            ok = lv >= 0
            out[q:q + W[v] * H[v], a][ok] = b.vals[b.ranges[gt[ok], 0] + lv[ok]]
        q += W[v] * H[v]
    return out


def test_brute_force_detects_a_tile_filter_that_is_not_conservative(orc, monkeypatch):
    # A planted mistake: tile levels one level too coarse.  The tiled render
    # then drops points some band pixels need, and the comparison above fails.
    rng = np.random.default_rng(21)
    sc = synth.uniform_scene(rng, 64, degree=3, log_scale=(-2.8, 0.5), dc_mode="coef")
    cams = synth.orbit_cameras(rng, 2, 3.0, [(32, 32), (48, 40)])
    f, _, _ = _small_fov(rng, sc.n, 2, cams)
    fa = orc.FovArrays.from_synth(f)
    rgb, _, _ = orc.render_brute(sc, cams, 16, fa)
    good = orc.tile_levels
    monkeypatch.setattr(orc, "tile_levels",
                        lambda c, t, fv: np.minimum(good(c, t, fv) + 1, fv.n_levels).astype(np.uint8))
    b = orc.bin_pairs(sc, cams, 16, fa)
    img = orc.render(sc, cams, 16, b, fa)
    assert np.abs(img.rgb - rgb).max() > 1e-6


def test_ambiguity_flags_cover_real_decision_flips(orc):
    # The oracle flags pixels whose alpha-floor or stop decision lies inside
    # the uncertainty window of an FP32 evaluation (alpha relative error below
    # 4e-5) and bounds what a flipped decision can change.  Scaling every
    # opacity by (1 + delta), |delta| below that error, flips exactly such
    # decisions in FP64: every pixel that moves by more than the continuous
    # change must be flagged, and move by no more than its bound.
    rng = np.random.default_rng(41)
    sc = synth.blob_scene(rng, 6000, n_blobs=8, degree=1, log_scale=(-3.2, 0.5))
    cams = synth.orbit_cameras(rng, 3, 3.0, [(96, 80), (64, 64), (128, 96)])
    b = orc.bin_pairs(sc, cams, 16)
    img = orc.render(sc, cams, 16, b)
    cont = 1e-4          # the continuous change of scaling alpha by |delta|
    n_jumped = 0
    for delta in (-3.5e-5, -2e-5, -1e-5, 1e-5, 2e-5, 3.5e-5):
        op2 = sc.opac.astype(np.float64) * (1.0 + delta)
        img2 = orc.render(sc, cams, 16, b, opac=op2)
        d = np.abs(img2.rgb - img.rgb).max(axis=1)
        jumped = d > cont
        n_jumped += int(jumped.sum())
        assert np.all(img.amb[jumped]), (delta, np.nonzero(jumped & ~img.amb)[0][:10])
        assert np.all(d <= img.ambB + cont), delta
    assert n_jumped > 0          # the perturbations do flip decisions here
    # the flags stay rare
    assert img.amb.mean() < 0.02, img.amb.mean()
    assert (img.T[:, 0] < 1e-2).mean() > 0.2      # many pixels reach the stop decision


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------
def test_input_order_invariance_and_bounds(orc):
    rng = np.random.default_rng(31)
    sc = synth.uniform_scene(rng, 300, degree=3, log_scale=(-3.0, 0.5), dc_mode="coef")
    cams = synth.camera_lookat((0, 0, -4), (0, 0, 0), 64, 64)[None]
    b = orc.bin_pairs(sc, cams, 16)
    img = orc.render(sc, cams, 16, b)
    depths = b.dbits[b.vis == 1]
    assert len(np.unique(depths)) == len(depths)
    perm = rng.permutation(sc.n)
    sp = synth.Scene(sc.means[perm], sc.scales[perm], sc.quats[perm], sc.opac[perm],
                     sc.sh[perm], sc.sh_degree)
    b2 = orc.bin_pairs(sp, cams, 16)
    img2 = orc.render(sp, cams, 16, b2)
    np.testing.assert_allclose(img2.rgb, img.rgb, atol=1e-14)
    np.testing.assert_array_equal(img2.last, img.last)
    # T stays in [1e-4, 1]; colour lies in [0, max c] (sum T_i alpha_i <= 1 - T)
    assert img.T[:, 0].min() >= 1e-4 and img.T[:, 0].max() <= 1.0
    vp = orc.project_values(sc, cams, b.vis)
    cmax = vp[b.vis == 1][:, orc.ORC_R:orc.ORC_B + 1].max()
    assert img.rgb.min() >= 0 and img.rgb.max() <= cmax + 1e-12
    # adding splats behind everything never raises the transmittance
    far = synth.uniform_scene(np.random.default_rng(32), 100, degree=3, log_scale=(-2.5, 0.3),
                              dc_mode="coef")
    far.means[:, 2] += 3.0
    sa = synth.Scene(*[np.concatenate([getattr(sc, k), getattr(far, k)])
                       for k in ("means", "scales", "quats", "opac", "sh")], 3)
    img3 = orc.render(sa, cams, 16, orc.bin_pairs(sa, cams, 16))
    assert np.all(img3.T[:, 0] <= img.T[:, 0] + 1e-15)


def test_stats_identities(orc):
    rng = np.random.default_rng(41)
    sc = synth.uniform_scene(rng, 500, degree=0, log_scale=(-3.2, 0.5))
    cams = synth.orbit_cameras(rng, 2, 4.0, [(64, 64), (48, 80)])
    b = orc.bin_pairs(sc, cams, 16)
    img = orc.render(sc, cams, 16, b, stats=True)
    tt, tu, pb, pd = img.stats
    assert tt.sum() == b.K                                   # Comp counts every pair
    assert pd.sum() == (img.last[:, 0] >= 0).sum()           # each blended pixel has one dominator
    assert np.all(tu <= tt) and np.all(pd <= pb)
    assert pb.sum() <= (img.last[:, 0] + 1).sum()            # blends <= list positions walked
    # per point, tiles_touched = kept pairs over all views
    np.testing.assert_array_equal(tt, b.counts.reshape(2, -1).sum(0))


# ---------------------------------------------------------------------------
# foveated render (Sec. 4.1 - 4.2)
# ---------------------------------------------------------------------------
def test_fov_all_points_in_all_levels_equals_plain(orc):
    rng = np.random.default_rng(51)
    sc = synth.uniform_scene(rng, 400, degree=0, log_scale=(-3.0, 0.5))
    cams = synth.orbit_cameras(rng, 2, 4.0, [(64, 64), (80, 48)])
    f, _, _ = _small_fov(rng, sc.n, 2, cams)
    f.bound_m[:] = 4
    fa = orc.FovArrays.from_synth(f)
    img_f = orc.render(sc, cams, 16, orc.bin_pairs(sc, cams, 16, fa), fa)
    img_p = orc.render(sc, cams, 16, orc.bin_pairs(sc, cams, 16))
    np.testing.assert_allclose(img_f.rgb, img_p.rgb, atol=1e-14)


def test_fov_far_gaze_reduces_to_outermost_level_subset(orc):
    rng = np.random.default_rng(52)
    sc = synth.uniform_scene(rng, 600, degree=0, log_scale=(-3.0, 0.5))
    cams = synth.camera_lookat((0, 0, -4), (0, 0, 0), 64, 64)[None]
    m = synth.nested_levels(rng, sc.n, 4)
    f = synth.Foveation(4, m, synth.ring_tangents([5, 10, 18]), 0.0,
                        np.array([[-1e4, -1e4]], np.float32))
    fa = orc.FovArrays.from_synth(f)
    img_f = orc.render(sc, cams, 16, orc.bin_pairs(sc, cams, 16, fa), fa)
    keep = m >= 4
    sub = synth.Scene(sc.means[keep], sc.scales[keep], sc.quats[keep], sc.opac[keep], sc.sh[keep], 0)
    img_s = orc.render(sub, cams, 16, orc.bin_pairs(sub, cams, 16))
    np.testing.assert_allclose(img_f.rgb, img_s.rgb, atol=1e-14)
    np.testing.assert_allclose(img_f.T[:, 0], img_s.T[:, 0], atol=1e-14)


def test_fov_levels_and_band_weights_by_geometry(orc):
    # One wide splat covers the image and each level has its own DC colour,
    # so colour / alpha at a pixel reveals its level and band weight.  Ring
    # radii 16/32/48 px (tan = 0.125, 0.25, 0.375 at f = 128: exact in
    # binary), band 8 px, gaze on a pixel centre.
    W = H = 128
    f = 128.0
    cams = axis_camera(W, H, f)
    sc = make_scene([[0, 0, 4.0]], [[6.0] * 3], opac=[0.5], sh=[[dc_for_rgb([0.2, 0.2, 0.2])]])
    cols = np.array([0.2, 0.4, 0.6, 0.8])
    dc_lv = np.stack([dc_for_rgb([c, c, c])[None, :] for c in cols[1:]])  # (3, 1, 3)
    gaze = np.array([[20.5, 60.5]], np.float32)
    fa = orc.FovArrays(4, np.array([4], np.uint8), np.array([0.125, 0.25, 0.375], np.float32),
                       8.0, gaze, None, None, dc_lv.astype(np.float32).astype(np.float64))
    b = orc.bin_pairs(sc, cams, 16, fa)
    img = orc.render(sc, cams, 16, b, fa)
    colf = cols.astype(np.float64)
    colf = (np.array([dc_for_rgb([c] * 3)[0] for c in cols]).astype(np.float32).astype(np.float64)
            * Y00 + 0.5)
    for d, lvl, w in [(5, 1, 1.0), (16, 2, 0.0), (20, 2, 0.5), (24, 2, 1.0), (30, 2, 1.0),
                      (34, 3, 0.25), (45, 3, 1.0), (50, 4, 0.25), (60, 4, 1.0), (90, 4, 1.0)]:
        q = 60 * W + 20 + d
        alpha = 1.0 - img.T[q, 0]
        assert alpha > 1 / 255
        assert img.wband[q] == pytest.approx(w, abs=1e-12)
        expect = colf[lvl - 1] if w == 1.0 else w * colf[lvl - 1] + (1 - w) * colf[lvl - 2]
        np.testing.assert_allclose(img.rgb[q, 0] / alpha, expect, rtol=1e-9)


def test_all_core_build_gives_identical_results(orc):
    # the -fopenmp build splits independent items and pixels over threads and
    # must not change a single bit (timed as the all-core CPU baseline)
    rng = np.random.default_rng(51)
    sc = synth.blob_scene(rng, 4000, n_blobs=6, degree=2, log_scale=(-3.2, 0.5))
    cams = synth.orbit_cameras(rng, 2, 3.0, [(96, 80), (64, 64)])
    pix = np.arange(0, 96 * 80 + 64 * 64, 7, dtype=np.int64)
    orc.use_all_cores(False)
    b1 = orc.bin_pairs(sc, cams, 16, tight=True)
    i1 = orc.render(sc, cams, 16, b1, pix=pix)
    try:
        if not orc.use_all_cores(True):
            pytest.skip("no OpenMP runtime")
        b2 = orc.bin_pairs(sc, cams, 16, tight=True)
        i2 = orc.render(sc, cams, 16, b2, pix=pix)
    finally:
        orc.use_all_cores(False)
    np.testing.assert_array_equal(b1.keys, b2.keys)
    np.testing.assert_array_equal(b1.vals, b2.vals)
    for a, b in ((i1.rgb, i2.rgb), (i1.T, i2.T), (i1.last, i2.last), (i1.ambB, i2.ambB)):
        np.testing.assert_array_equal(a, b)
