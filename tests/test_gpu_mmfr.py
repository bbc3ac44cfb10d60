"""Foveated render with a separate model per quality level
(GS_FLAG_MULTI_MODEL, Sec. 4.1 main pipeline) on the GPU against the FP64
oracle: binning bit-exact, images within the forward tolerance (blend bands
included), gradients within 1e-3, and the entry points' argument checks."""
import numpy as np
import pytest

from paper_2407_00435_gb300 import synth
from helpers import compare_images, run_gpu
from helpers import compare_grads as _compare
from test_gpu_forward import check_bins_exact, gpu_bins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_00435_gb300 import gs as _gs
    return _gs


def _workload(seed, n, sizes, tile=16, L=3, rings=(6.0, 12.0), band=6.0, degree=1):
    rng = np.random.default_rng(seed)
    base = synth.blob_scene(rng, n, n_blobs=8, degree=degree, log_scale=(-3.0, 0.5))
    cams = synth.orbit_cameras(rng, len(sizes), 3.0, sizes)
    m = synth.nested_levels(rng, n, L)
    sc, lv = synth.multi_model_scene(rng, base, m, L)
    f = synth.Foveation(L, lv, synth.ring_tangents(list(rings)), band,
                        synth.random_gaze(rng, cams), disjoint=True)
    return synth.Workload("mmfr", sc, cams, tile, f)


@pytest.mark.parametrize("tile,tight", [(16, False), (16, True), (8, False), (8, True)])
def test_mmfr_forward_matches_oracle(gs, orc, tile, tight):
    wl = _workload(61, 4000, [(112, 96), (80, 72)], tile=tile)
    r, out, _, _ = run_gpu(gs, wl, fov=wl.fov, tile=tile, tight=tight, multi_model=True,
                           bg=(0.1, 0.2, 0.3))
    fa = orc.FovArrays.from_synth(wl.fov)
    ob = orc.bin_pairs(wl.scene, wl.cams, tile, fa, tight=tight)
    img = orc.render(wl.scene, wl.cams, tile, ob, fa, bg=(0.1, 0.2, 0.3))
    check_bins_exact(gpu_bins(gs, r), ob, wl.scene.n)
    assert (img.wband < 1.0).sum() > 100          # blend bands are exercised
    compare_images(out["rgb"].cpu().numpy(), img)


def test_mmfr_stats_and_plain_view(gs, orc):
    """A plain view in a multi-model call renders model 1 only; the
    statistics render counts the same blends as the oracle."""
    wl = _workload(62, 3000, [(96, 80), (64, 64)])
    wl.fov.view_fov = np.array([1, 0], np.uint8)
    r, out, _, _ = run_gpu(gs, wl, fov=wl.fov, multi_model=True, stats=True)
    fa = orc.FovArrays.from_synth(wl.fov)
    ob = orc.bin_pairs(wl.scene, wl.cams, wl.tile, fa)
    img = orc.render(wl.scene, wl.cams, wl.tile, ob, fa, stats=True)
    compare_images(out["rgb"].cpu().numpy(), img)
    st = out["stats"].cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(st[0], img.stats[0])        # tiles touched
    # plain view: the level-1 model alone, as a plain render of that model
    lv = wl.fov.bound_m
    sel = np.nonzero(lv == 1)[0]
    sub = synth.Scene(wl.scene.means[sel], wl.scene.scales[sel], wl.scene.quats[sel],
                      wl.scene.opac[sel], wl.scene.sh[sel], wl.scene.sh_degree)
    cam1 = wl.cams[1:2]
    b1 = orc.bin_pairs(sub, cam1, wl.tile)
    i1 = orc.render(sub, cam1, wl.tile, b1)
    p0 = int(wl.cams[0, 16]) * int(wl.cams[0, 17])
    compare_images(out["rgb"].cpu().numpy()[p0:], i1)


def test_mmfr_backward_matches_oracle(gs, orc):
    import torch
    wl = _workload(63, 2500, [(96, 96), (80, 64)], L=4, rings=(5.0, 10.0, 16.0))
    sc = gs.scene_to_device(wl.scene)
    f = gs.fov_to_device(wl.fov)
    r = gs.Renderer(wl.scene.n, wl.scene.sh_degree, wl.cams, multi_model=True, backward=True)
    r.fit(sc, f)
    out = r.alloc_outputs(fov=True)
    r.render(out, fov=True)
    fa = orc.FovArrays.from_synth(wl.fov)
    ob = orc.bin_pairs(wl.scene, wl.cams, wl.tile, fa)
    img = orc.render(wl.scene, wl.cams, wl.tile, ob, fa)
    dL = np.random.default_rng(7).uniform(-1, 1, (r.P, 3))
    dL[img.margin < 1e-3] = 0.0
    S = (wl.scene.sh_degree + 1) ** 2
    n = wl.scene.n
    g = {k: torch.empty(s, device="cuda") for k, s in
         (("means", (n, 3)), ("scales", (n, 3)), ("quats", (n, 4)), ("opac", (n,)),
          ("sh", (n, S, 3)))}
    r.backward(torch.from_numpy(dL.astype(np.float32)).cuda(), out, g)
    code, c = r.counters()
    assert code == gs.GS_OK, c
    ref = orc.backward(wl.scene, wl.cams, wl.tile, ob, dL.astype(np.float32).astype(np.float64), fa)
    for k, rk in (("means", ref.means), ("scales", ref.scales), ("quats", ref.quats),
                  ("opac", ref.opac), ("sh", ref.sh)):
        _compare(k, g[k].cpu().numpy(), rk, ref.mag[k])


def test_mmfr_argument_checks(gs):
    wl = _workload(64, 500, [(64, 48)])
    sc = gs.scene_to_device(wl.scene)
    r = gs.Renderer(wl.scene.n, wl.scene.sh_degree, wl.cams, multi_model=True)
    with pytest.raises(gs.GsError):
        r.project(sc)                                  # the levels select the models
    op, dc = synth.multiversion_params(np.random.default_rng(1), wl.scene, 3)
    with pytest.raises(gs.GsError):
        r.project(sc, gs.fov_to_device(wl.fov, opacity_lv=op))   # every model has its own
    r.fit(sc, gs.fov_to_device(wl.fov))
    out = r.alloc_outputs(fov=True)
    with pytest.raises(gs.GsError):
        r.render(out)                                  # plain render of a multi-model plan
    r.render(out, fov=True)
