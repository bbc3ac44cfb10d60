"""CUDA HVSQ (gs_hvsq) against the FP64 reference of oracle/hvsq.py: the HVSQ
of every quality region and the gradient element by element, on images
whose poolings span one pixel to beyond the image, flat regions (std 0),
ragged sizes; at full size, properties that hold at any size (symmetry,
shift invariance, zero at equal images, the directional derivative)."""
import numpy as np
import pytest

from oracle import hvsq as H
from paper_2407_00435_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_00435_gb300 import gs as _gs
    return _gs


def _images(rng, h, w, flat=False):
    ref = rng.uniform(0, 1, (h, w, 3)).astype(np.float32)
    alt = np.clip(ref + rng.normal(0, 0.08, ref.shape), 0, 1.2).astype(np.float32)
    if flat:
        ref[: h // 3] = 0.25
        alt[: h // 3] = 0.4
    return alt, ref


def _oracle_regions(w, h, gaze, focal, ring_tan):
    f32 = np.float32
    ys, xs = np.mgrid[0:h, 0:w]
    dx = (xs.astype(f32) + f32(0.5)) - f32(gaze[0])
    dy = (ys.astype(f32) + f32(0.5)) - f32(gaze[1])
    d2 = dx * dx + dy * dy
    g = np.zeros((h, w), np.int64)
    for t in np.asarray(ring_tan, f32):
        R = f32(focal) * t
        g += (d2 >= R * R).astype(np.int64)
    return g


def _run(gs, alt, ref, gaze, focal, ring_tan, pool_tan, r_base):
    import torch
    h, w, _ = alt.shape
    v = gs.HvsqView(w, h, gaze, focal, ring_tan, pool_tan, r_base)
    a = torch.from_numpy(alt.reshape(-1, 3)).cuda()
    r = torch.from_numpy(ref.reshape(-1, 3)).cuda()
    out = torch.empty(v.n_regions, dtype=torch.float64, device="cuda")
    grad = torch.empty_like(a)
    v(a, r, out, grad)
    out2 = torch.empty_like(out)
    v(a, r, out2)                      # forward only: the same values (to the order of
    torch.cuda.synchronize()           # the FP64 atomic sums)
    np.testing.assert_allclose(out.cpu().numpy(), out2.cpu().numpy(), rtol=1e-12)
    return out.cpu().numpy(), grad.cpu().numpy().reshape(h, w, 3)


@pytest.mark.parametrize("case", ["rings", "ragged_flat", "one_pixel_poolings", "huge_poolings"])
def test_hvsq_and_gradient_match_oracle(gs, case):
    rng = np.random.default_rng({"rings": 1, "ragged_flat": 2, "one_pixel_poolings": 3,
                                 "huge_poolings": 4}[case])
    h, w = (80, 96) if case != "ragged_flat" else (37, 53)
    alt, ref = _images(rng, h, w, flat=case == "ragged_flat")
    gaze = (w * 0.4, h * 0.55)
    focal = 30.0
    ring_tan = synth.ring_tangents([20, 40, 60]) if case != "one_pixel_poolings" else np.zeros(0, np.float32)
    if case == "one_pixel_poolings":
        pool_tan, r_base = np.zeros(0, np.float32), 0
    elif case == "huge_poolings":
        pool_tan, r_base = synth.pooling_tangents(20.0, 0.5, 64)
    else:
        pool_tan, r_base = synth.pooling_tangents(1.0, 0.004, 12)
    got, g = _run(gs, alt, ref, gaze, focal, ring_tan, pool_tan, r_base)
    rad = H.pooling_radius(w, h, gaze, focal, pool_tan, r_base)
    reg = _oracle_regions(w, h, gaze, focal, ring_tan)
    nreg = len(ring_tan) + 1
    want = H.hvsq(alt.astype(np.float64), ref.astype(np.float64), rad, reg, nreg)
    wg = H.hvsq_grad(alt.astype(np.float64), ref.astype(np.float64), rad, reg, nreg)
    if case != "one_pixel_poolings":
        assert rad.max() > rad.min()                  # poolings of several sizes
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-15)
    # gradient: FP64 arithmetic rounded to FP32 once
    np.testing.assert_allclose(g, wg, rtol=2e-6, atol=1e-6 * np.abs(wg).max())
    print(f"[hvsq {case}] regions {got}, max |grad - ref| {np.abs(g - wg).max():.3g} "
          f"of max {np.abs(wg).max():.3g}")


def test_full_size_properties(gs):
    # the foveated stereo eye's geometry (1920 x 1920, 60 deg field of view,
    # rings at 10/20/35 deg, the workload pooling law r = floor(1 + 0.025 e^2))
    import torch
    rng = np.random.default_rng(7)
    h = w = 1920
    ref = rng.uniform(0, 1, (h * w, 3)).astype(np.float32)
    alt = np.clip(ref + rng.normal(0, 0.05, ref.shape), 0, 1).astype(np.float32)
    focal = 0.5 * h / np.tan(np.radians(30.0))
    pool_tan, r_base = synth.pooling_tangents()
    v = gs.HvsqView(w, h, (800.0, 1100.0), focal, synth.ring_tangents([10, 20, 35]), pool_tan,
                    r_base)
    a = torch.from_numpy(alt).cuda()
    r = torch.from_numpy(ref).cuda()
    out = torch.empty(4, dtype=torch.float64, device="cuda")

    def hv(x, y, grad=None):
        v(x, y, out, grad)
        return out.cpu().numpy().copy()

    g = torch.empty_like(a)
    base = hv(a, r, g)
    assert np.all(base > 0)
    np.testing.assert_allclose(hv(r, a), base, rtol=1e-9)            # symmetric
    np.testing.assert_allclose(hv(a + 0.125, r + 0.125), base, rtol=1e-6)   # shift
    zg = torch.empty_like(a)
    assert np.all(hv(a, a, zg) == 0.0) and float(zg.abs().max()) == 0.0
    # directional derivative of the summed loss along a random direction
    d = torch.from_numpy(rng.normal(0, 1, alt.shape).astype(np.float32)).cuda()
    eps = 1e-3
    fd = (hv(a + eps * d, r).sum() - hv(a - eps * d, r).sum()) / (2 * eps)
    an = float((g.double() * d.double()).sum())
    assert abs(fd - an) <= 1e-4 * abs(an), (fd, an)
