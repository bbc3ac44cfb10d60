"""Opacity-aware tight support on the GPU: the kept tile pairs, their order
and the per-tile ranges equal the FP32 oracle's bit for bit, and images
match the FP64 oracle as with the full 3-sigma rectangles."""
import numpy as np
import pytest

from paper_2407_00435_gb300 import synth
from helpers import compare_grads, compare_images, run_gpu
from test_gpu_forward import check_bins_exact, gpu_bins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_00435_gb300 import gs as _gs
    return _gs


def test_tight_plain_bins_exact_and_image(gs, orc):
    wl = synth.workload(0)
    r, out, _, _ = run_gpu(gs, wl, tight=True, stats=True)
    ob = orc.bin_pairs(wl.scene, wl.cams, 16, tight=True)
    ob_rect = orc.bin_pairs(wl.scene, wl.cams, 16)
    assert ob.K < ob_rect.K
    check_bins_exact(gpu_bins(gs, r), ob, wl.scene.n)
    img = orc.render(wl.scene, wl.cams, 16, ob, stats=True)
    compare_images(out["rgb"].cpu().numpy(), img)
    amb = img.amb
    assert np.array_equal(out["last"].cpu().numpy()[~amb], img.last[~amb, 0])
    st = out["stats"].cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(st[0], img.stats[0])      # tiles touched = kept pairs


def test_tight_ragged_multiview_tile8(gs, orc):
    rng = np.random.default_rng(4141)
    sc = synth.blob_scene(rng, 6000, n_blobs=8, degree=2, log_scale=(-3.2, 0.6))
    sc.opac[:500] = rng.uniform(1 / 255, 0.02, 500).astype(np.float32)
    cams = synth.orbit_cameras(rng, 3, 3.5, [(101, 37), (64, 80), (133, 90)])
    for tile in (16, 8):
        wl = synth.Workload("tight_ragged", sc, cams, tile)
        r, out, _, _ = run_gpu(gs, wl, tight=True, bg=(0.3, 0.2, 0.1))
        ob = orc.bin_pairs(sc, cams, tile, tight=True)
        check_bins_exact(gpu_bins(gs, r), ob, sc.n)
        compare_images(out["rgb"].cpu().numpy(), orc.render(sc, cams, tile, ob, bg=(0.3, 0.2, 0.1)))


@pytest.mark.parametrize("mv", [False, True])
def test_tight_foveated(gs, orc, mv):
    rng = np.random.default_rng(4242)
    sc = synth.blob_scene(rng, 15000, n_blobs=12, degree=1)
    cams = synth.orbit_cameras(rng, 2, 3.0, [(144, 128), (96, 112)])
    m = synth.nested_levels(rng, sc.n, 4)
    f = synth.Foveation(4, m, synth.ring_tangents([6, 12, 20]), 8.0, synth.random_gaze(rng, cams),
                        np.array([1, 0], np.uint8))
    mvp = synth.multiversion_params(rng, sc, 4) if mv else None
    if mv:   # some level opacities above the base one widen the support
        mvp = (np.ascontiguousarray(mvp[0], np.float32), mvp[1])
        mvp[0][:, : sc.n // 4] = 0.97
    wl = synth.Workload("tight_fov", sc, cams, 16, f)
    r, out, _, _ = run_gpu(gs, wl, fov=f, mv=mvp, tight=True)
    fa = orc.FovArrays.from_synth(f, *(mvp or (None, None)))
    ob = orc.bin_pairs(sc, cams, 16, fa, tight=True)
    check_bins_exact(gpu_bins(gs, r), ob, sc.n)
    img = orc.render(sc, cams, 16, ob, fa)
    compare_images(out["rgb"].cpu().numpy(), img)


def test_tight_backward_matches_oracle(gs, orc):
    import torch
    rng = np.random.default_rng(4343)
    sc = synth.blob_scene(rng, 3000, n_blobs=6, degree=2, log_scale=(-3.0, 0.5))
    cams = synth.orbit_cameras(rng, 2, 3.0, [(96, 80), (64, 64)])
    d = gs.scene_to_device(sc)
    r = gs.Renderer(sc.n, sc.sh_degree, cams, backward=True, tight=True)
    r.fit(d)
    out = r.alloc_outputs()
    r.render(out)
    ob = orc.bin_pairs(sc, cams, 16, tight=True)
    img = orc.render(sc, cams, 16, ob)
    dL = rng.uniform(-1, 1, (r.P, 3))
    dL[img.margin < 1e-3] = 0.0
    S = (sc.sh_degree + 1) ** 2
    g = {k: torch.empty(s, device="cuda") for k, s in
         (("means", (sc.n, 3)), ("scales", (sc.n, 3)), ("quats", (sc.n, 4)), ("opac", (sc.n,)),
          ("sh", (sc.n, S, 3)))}
    r.backward(torch.from_numpy(dL.astype(np.float32)).cuda(), out, g)
    assert r.counters()[0] == gs.GS_OK
    ref = orc.backward(sc, cams, 16, ob, dL.astype(np.float32).astype(np.float64))
    for k, rk in (("means", ref.means), ("scales", ref.scales), ("quats", ref.quats),
                  ("opac", ref.opac), ("sh", ref.sh)):
        compare_grads(k, g[k].cpu().numpy(), rk, ref.mag[k])


def test_tight_full_size_1080p_bins_exact_and_sampled_pixels(gs, orc):
    wl = synth.workload(1)
    r, out, _, _ = run_gpu(gs, wl, tight=True)
    ob = orc.bin_pairs(wl.scene, wl.cams, 16, tight=True)
    check_bins_exact(gpu_bins(gs, r), ob, wl.scene.n)
    rng = np.random.default_rng(6)
    pix = np.array(sorted(set(rng.choice(1920 * 1080, 3000, replace=False))), np.int64)
    img = orc.render(wl.scene, wl.cams, 16, ob, pix=pix)
    compare_images(out["rgb"].cpu().numpy()[pix], img)
