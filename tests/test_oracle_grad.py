"""The oracle's analytic FP64 gradient against central finite differences of
the oracle's own FP64 forward pass (binning held fixed).

A parameter whose +-h perturbation flips a discrete decision (alpha floor,
early stop, colour clamp) shows a jump; such parameters are detected by
comparing the difference quotient at h and h/2 and are left out (and
counted).  Sub-case of the forward+backward workload: 64 points, 32x32.
"""
import numpy as np
import pytest

from paper_2407_00435_gb300 import synth


def _loss(orc, sc, cams, bins, dL, fa, params, tile=16):
    m, s, q, o, h = params["means"], params["scales"], params["quats"], params["opac"], params["sh"]
    vp = orc.project_values(sc, cams, bins.vis, means=m, scales=s, quats=q, sh=h)
    fa2 = fa
    if fa is not None and ("opac_lv" in params or "dc_lv" in params):
        fa2 = orc.FovArrays(fa.n_levels, fa.bound_m, fa.ring_tan, fa.band_px, fa.gaze,
                            fa.view_fov, params.get("opac_lv", fa.opacity_lv),
                            params.get("dc_lv", fa.dc_lv))
    img = orc.render(sc, cams, tile, bins, fa2, vp=vp, opac=o)
    return float((img.rgb * dL).sum())


def _check(orc, sc, cams, fa, seed):
    rng = np.random.default_rng(seed)
    bins = orc.bin_pairs(sc, cams, 16, fa)
    W, H, _, _ = orc.view_dims(cams, 16)
    P = int((W * H).sum())
    dL = rng.uniform(-1, 1, (P, 3))
    g = orc.backward(sc, cams, 16, bins, dL, fa)
    base = {"means": sc.means.astype(np.float64), "scales": sc.scales.astype(np.float64),
            "quats": sc.quats.astype(np.float64), "opac": sc.opac.astype(np.float64),
            "sh": sc.sh.astype(np.float64)}
    analytic = {"means": g.means, "scales": g.scales, "quats": g.quats, "opac": g.opac,
                "sh": g.sh}
    if fa is not None and fa.opacity_lv is not None:
        base["opac_lv"] = fa.opacity_lv.copy()
        analytic["opac_lv"] = g.opac_lv
    if fa is not None and fa.dc_lv is not None:
        base["dc_lv"] = fa.dc_lv.copy()
        analytic["dc_lv"] = g.dc_lv
    vp0 = orc.project_values(sc, cams, bins.vis)
    img0 = orc.render(sc, cams, 16, bins, fa, vp=vp0)
    absL = float(np.abs(img0.rgb * dL).sum()) + 1.0   # scale of the loss's rounding error
    n_cmp = n_skip = 0
    for name, arr in base.items():
        flat = arr.reshape(-1)
        an = analytic[name].reshape(-1)
        fds = np.zeros_like(flat)
        ok = np.zeros(flat.shape, bool)
        noise = np.zeros_like(flat)
        for k in range(flat.size):
            x = flat[k]
            h = 1e-5 * max(abs(x), 1e-2)

            def L_at(val):
                p = {kk: vv.copy() for kk, vv in base.items()}
                p[name].reshape(-1)[k] = val
                return _loss(orc, sc, cams, bins, dL, fa, p)
            f1 = (L_at(x + h) - L_at(x - h)) / (2 * h)
            f2 = (L_at(x + h / 2) - L_at(x - h / 2)) / h
            fds[k] = f1
            noise[k] = 1e-13 * absL / h
            ok[k] = abs(f1 - f2) <= 1e-4 * abs(f1) + 10 * noise[k]
        scale = np.abs(fds[ok]).max() if ok.any() else 1.0
        err = np.abs(an[ok] - fds[ok])
        tol = 1e-3 * np.abs(fds[ok]) + 1e-7 * scale + 10 * noise[ok]
        bad = np.nonzero(err > tol)[0]
        assert len(bad) == 0, (name, an[ok][bad][:5], fds[ok][bad][:5])
        n_cmp += int(ok.sum())
        n_skip += int((~ok).sum())
    return n_cmp, n_skip


def test_gradient_plain_matches_fd(orc):
    rng = np.random.default_rng(1003)
    sc = synth.blob_scene(rng, 64, n_blobs=4, degree=3, log_scale=(-2.6, 0.4), opac_std=1.5)
    cams = synth.camera_lookat((0.4, -0.3, -3.5), (0, 0, 0), 32, 32)[None]
    n_cmp, n_skip = _check(orc, sc, cams, None, 7)
    assert n_cmp > 0.9 * (n_cmp + n_skip)


def test_gradient_foveated_multiversion_matches_fd(orc):
    rng = np.random.default_rng(2003)
    sc = synth.blob_scene(rng, 48, n_blobs=3, degree=1, log_scale=(-2.6, 0.4), opac_std=1.5)
    cams = synth.orbit_cameras(rng, 2, 3.5, [(32, 32), (40, 24)])
    m = synth.nested_levels(rng, sc.n, 3)
    gaze = np.array([[16.0, 16.0], [10.0, 12.0]], np.float32)
    f = synth.Foveation(3, m, np.array([0.08, 0.2], np.float32), 6.0, gaze)
    op, dc = synth.multiversion_params(rng, sc, 3)
    fa = orc.FovArrays.from_synth(f, op, dc)
    n_cmp, n_skip = _check(orc, sc, cams, fa, 8)
    assert n_cmp > 0.9 * (n_cmp + n_skip)


@pytest.mark.parametrize("fov_mode", [False, True])
def test_term_magnitudes_bound_every_gradient_element(orc, fov_mode):
    # Grads.mag is the chain with every term in absolute value: by the
    # triangle inequality it bounds |gradient| element by element (the GPU
    # parity bound scales with it), and it exceeds the gradient where terms
    # cancel, e.g. the quaternion of a needle-shaped point.
    rng = np.random.default_rng(3100 + fov_mode)
    sc = synth.blob_scene(rng, 400, n_blobs=5, degree=2, log_scale=(-3.0, 0.6))
    cams = synth.orbit_cameras(rng, 2, 3.0, [(48, 40), (32, 32)])
    fa = None
    if fov_mode:
        m = synth.nested_levels(rng, sc.n, 3)
        f = synth.Foveation(3, m, synth.ring_tangents([5, 10]), 6.0, synth.random_gaze(rng, cams))
        op, dc = synth.multiversion_params(rng, sc, 3)
        fa = orc.FovArrays.from_synth(f, op, dc)
    bins = orc.bin_pairs(sc, cams, 16, fa)
    W, H, _, _ = orc.view_dims(cams, 16)
    dL = rng.uniform(-1, 1, (int((W * H).sum()), 3))
    g = orc.backward(sc, cams, 16, bins, dL, fa)
    groups = {"means": g.means, "scales": g.scales, "quats": g.quats, "opac": g.opac, "sh": g.sh}
    if fov_mode:
        groups.update(opac_lv=g.opac_lv, dc_lv=g.dc_lv)
    for k, v in groups.items():
        mag = g.mag[k]
        assert np.all(np.abs(v) <= mag * (1 + 1e-9) + 1e-300), k
        assert (mag > 0).any(), k
    # cancellation shows: somewhere the terms are far larger than their sum
    assert (g.mag["quats"] > 10 * np.abs(g.quats)).any()


def test_term_magnitude_of_a_single_term_is_its_value(orc):
    # one isotropic point, one pixel with a loss weight: d_opac is one term,
    # so its magnitude equals its absolute value
    W = H = 16
    row = np.zeros(20, np.float32)
    row[[0, 4, 8]] = 1.0
    row[12:20] = [20.0, 20.0, W / 2, H / 2, W, H, 0.2, 1000.0]
    cams = row[None]
    sc = synth.Scene(np.array([[0.0, 0.0, 3.0]], np.float32), np.full((1, 3), 0.05, np.float32),
                     np.array([[1.0, 0.0, 0.0, 0.0]], np.float32), np.array([0.5], np.float32),
                     np.full((1, 1, 3), 0.4, np.float32), 0)
    bins = orc.bin_pairs(sc, cams, 16)
    dL = np.zeros((W * H, 3))
    dL[8 * W + 8] = [0.0, -0.7, 0.0]     # one channel, black background: one term
    g = orc.backward(sc, cams, 16, bins, dL)
    assert abs(g.opac[0]) > 0
    np.testing.assert_allclose(g.mag["opac"][0], abs(g.opac[0]), rtol=1e-12)
