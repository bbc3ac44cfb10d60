"""Parity at the full sizes of the foveated, backward and batched workloads,
in the plan options the benchmark times them with:

* foveated stereo: 3M points, 2 eyes at 1920x1920, 4 nested levels, rings at
  10/20/35 degrees, 32-px blend band, tight support -- binning bit-exact and
  sampled pixels, a third of them inside blend bands or on ring boundaries;
* forward + backward: 500k points, SH3, 1024x1024 views on the orbit (two of
  the eight), tight support, the L1 loss against seeded uniform targets --
  gradients element by element, tiles longer than one 256-point batch;
* the 64-view batch: 6M points (600 blobs), a subset of its views (a
  2048x2048 foveated, a 256x256 plain and two more) under the autotuned plan
  (16-px tiles, 7-bit pair-sort digits, whole tiles) -- binning bit-exact and
  sampled pixels of every view.
The oracle is FP64 on the host; these run for minutes."""
import numpy as np
import pytest

from paper_2407_00435_gb300 import synth
from helpers import compare_grads, compare_images
from test_gpu_forward import check_bins_exact, gpu_bins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_00435_gb300 import gs as _gs
    return _gs


def _pixel_rings(cams, fov, v):
    """Distance of view v's pixel centres to its gaze and the ring radii."""
    W, H = int(cams[v, 16]), int(cams[v, 17])
    fy = float(cams[v, 13])
    ys, xs = np.divmod(np.arange(W * H), W)
    d = np.hypot(xs + 0.5 - fov.gaze[v, 0], ys + 0.5 - fov.gaze[v, 1])
    R = fy * np.asarray(fov.ring_tan, np.float64)
    return d, R


def test_foveated_stereo_full_size(gs, orc):
    import torch
    wl = synth.workload(2)
    sc = gs.scene_to_device(wl.scene)
    f = gs.fov_to_device(wl.fov)
    r = gs.Renderer(wl.scene.n, 3, wl.cams, foveated=True, tight=True)
    r.fit(sc, f)
    out = r.alloc_outputs(fov=True)
    r.render(out, fov=True)
    torch.cuda.synchronize()
    fa = orc.FovArrays.from_synth(wl.fov)
    ob = orc.bin_pairs(wl.scene, wl.cams, 16, fa, tight=True)
    check_bins_exact(gpu_bins(gs, r), ob, wl.scene.n)
    tl = r.region(gs.GS_REGION_TILE_LEVEL, torch.uint8, r.T_tiles).cpu().numpy()
    np.testing.assert_array_equal(tl, ob.tile_level)
    rng = np.random.default_rng(22)
    P1 = 1920 * 1920
    pix, n_band, n_edge = [], 0, 0
    for v in range(2):
        d, R = _pixel_rings(wl.cams, wl.fov, v)
        band = np.zeros(P1, bool)
        edge = np.zeros(P1, bool)
        for Rk in R:
            band |= (d >= Rk) & (d < Rk + wl.fov.band_px)
            edge |= np.abs(d - Rk) < 1.0
        b = rng.choice(np.nonzero(band)[0], 400, replace=False)
        e = rng.choice(np.nonzero(edge)[0], 200, replace=False)
        u = rng.choice(P1, 1100, replace=False)
        n_band += len(b)
        n_edge += len(e)
        pix += list(v * P1 + np.concatenate([b, e, u]))
    pix = np.array(sorted(set(pix)), np.int64)
    assert len(pix) >= 3000 and n_band + n_edge >= 1000
    img = orc.render(wl.scene, wl.cams, 16, ob, fa, pix=pix)
    assert (img.wband < 1).sum() >= 800          # pixels that blend two levels
    compare_images(out["rgb"].cpu().numpy()[pix], img, label="foveated stereo 2x1920^2 3M")


@pytest.mark.parametrize("foveated", [False, True])
def test_backward_full_size_views(gs, orc, foveated):
    # foveated: the views as the foveated forward + backward of the benchmark
    # time them (4 nested levels, rings at 10/20/35 degrees, 32-px band)
    import torch
    wl = synth.fov_fwd_bwd_workload() if foveated else synth.workload(3)
    cams = wl.cams[:2]
    fov = fa = f = None
    if foveated:
        fov = synth.Foveation(wl.fov.n_levels, wl.fov.bound_m, wl.fov.ring_tan,
                              wl.fov.band_px, wl.fov.gaze[:2])
        f = gs.fov_to_device(fov)
        fa = orc.FovArrays.from_synth(fov)
    sc = gs.scene_to_device(wl.scene)
    r = gs.Renderer(wl.scene.n, 3, cams, backward=True, tight=True, foveated=foveated)
    r.fit(sc, f)
    out = r.alloc_outputs(fov=foveated)
    r.render(out, fov=foveated)
    torch.cuda.synchronize()
    ob = orc.bin_pairs(wl.scene, cams, 16, fa, tight=True)
    lens = ob.ranges[:, 1].astype(np.int64) - ob.ranges[:, 0]
    assert lens.max() > 256 and (lens > 256).sum() > 100   # tiles span several staging batches
    img = orc.render(wl.scene, cams, 16, ob, fa)
    if foveated:
        assert (img.wband < 1).mean() > 0.01     # pixels blending two levels
    rgb = out["rgb"].cpu().numpy()
    rng = np.random.default_rng(1003)
    target = rng.uniform(0, 1, (8 * 1024 * 1024, 3)).astype(np.float32)[:r.P]
    diff = rgb.astype(np.float64) - target
    # L1 loss: dL/drgb = sign / numel; pixels whose sign or decisions are
    # uncertain are left out on both sides
    keep = (img.margin >= 1e-3) & (np.abs(img.rgb - target).min(axis=1) > 1e-3)
    assert keep.mean() > 0.95
    dL = (np.sign(diff) / diff.size * keep[:, None]).astype(np.float32)
    S = 16
    g = {k: torch.empty(s, device="cuda") for k, s in
         (("means", (wl.scene.n, 3)), ("scales", (wl.scene.n, 3)), ("quats", (wl.scene.n, 4)),
          ("opac", (wl.scene.n,)), ("sh", (wl.scene.n, S, 3)))}
    r.backward(torch.from_numpy(dL).cuda(), out, g)
    assert r.counters()[0] == gs.GS_OK
    ref = orc.backward(wl.scene, cams, 16, ob, dL.astype(np.float64), fa)
    for k, rk in (("means", ref.means), ("scales", ref.scales), ("quats", ref.quats),
                  ("opac", ref.opac), ("sh", ref.sh)):
        compare_grads(k, g[k].cpu().numpy(), rk, ref.mag[k])


def test_batched_views_full_size_subset_autotuned_plan(gs, orc):
    import torch
    wl = synth.workload(4)
    sides = wl.cams[:, 16].astype(int)
    vf = wl.fov.view_fov
    pick = [int(np.nonzero((sides == 2048) & (vf == 1))[0][0]),
            int(np.nonzero((sides == 256) & (vf == 0))[0][0]),
            int(np.nonzero((sides == 512) & (vf == 1))[0][0]),
            int(np.nonzero((sides == 1024) & (vf == 0))[0][0])]
    cams = wl.cams[pick]
    fov = synth.Foveation(wl.fov.n_levels, wl.fov.bound_m, wl.fov.ring_tan, wl.fov.band_px,
                          wl.fov.gaze[pick], vf[pick])
    sc = gs.scene_to_device(wl.scene)
    f = gs.fov_to_device(fov)
    r = gs.Renderer(wl.scene.n, 3, cams, foveated=True, tight=True, tile=16, radix_bits=7,
                    chunk=0)
    r.fit(sc, f)
    out = r.alloc_outputs(fov=True)
    r.render(out, fov=True)
    torch.cuda.synchronize()
    fa = orc.FovArrays.from_synth(fov)
    ob = orc.bin_pairs(wl.scene, cams, 16, fa, tight=True)
    check_bins_exact(gpu_bins(gs, r), ob, wl.scene.n)
    rng = np.random.default_rng(44)
    base = np.concatenate([[0], np.cumsum(cams[:, 16].astype(np.int64) * cams[:, 17].astype(np.int64))])
    pix = np.concatenate([base[v] + rng.choice(base[v + 1] - base[v], 800, replace=False)
                          for v in range(4)])
    pix = np.sort(pix)
    img = orc.render(wl.scene, cams, 16, ob, fa, pix=pix)
    compare_images(out["rgb"].cpu().numpy()[pix], img, label="64-view batch subset")
