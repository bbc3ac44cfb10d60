"""CUDA backward vs the FP64 oracle's analytic gradient (itself pinned to
FP64 finite differences in test_oracle_grad.py): relative error 1e-3 per
parameter group, through the C ABI and through torch.autograd."""
import numpy as np
import pytest

from paper_2407_00435_gb300 import synth

from helpers import compare_grads as _compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_00435_gb300 import gs as _gs
    return _gs


def _run(gs, orc, wl, fov=None, mv=None, seed=0):
    import torch
    sc = gs.scene_to_device(wl.scene)
    f = gs.fov_to_device(fov, opacity_lv=None if mv is None else mv[0],
                         dc_lv=None if mv is None else mv[1]) if fov is not None else None
    r = gs.Renderer(wl.scene.n, wl.scene.sh_degree, wl.cams, foveated=fov is not None,
                    backward=True)
    r.fit(sc, f)
    out = r.alloc_outputs(fov=fov is not None)
    r.render(out, fov=fov is not None)
    fa = orc.FovArrays.from_synth(fov, *(mv or (None, None))) if fov is not None else None
    ob = orc.bin_pairs(wl.scene, wl.cams, wl.tile, fa)
    img = orc.render(wl.scene, wl.cams, wl.tile, ob, fa)
    rng = np.random.default_rng(seed)
    dL = rng.uniform(-1, 1, (r.P, 3))
    dL[img.margin < 1e-3] = 0.0     # keep decision-ambiguous pixels out of the loss
    dL32 = torch.from_numpy(dL.astype(np.float32)).cuda()
    S = (wl.scene.sh_degree + 1) ** 2
    g = {k: torch.empty(s, device="cuda") for k, s in
         (("means", (wl.scene.n, 3)), ("scales", (wl.scene.n, 3)), ("quats", (wl.scene.n, 4)),
          ("opac", (wl.scene.n,)), ("sh", (wl.scene.n, S, 3)))}
    if mv is not None:
        g["opac_lv"] = torch.empty(mv[0].shape, device="cuda")
        g["dc_lv"] = torch.empty(mv[1].shape, device="cuda")
    r.backward(dL32, out, g)
    code, c = r.counters()
    assert code == gs.GS_OK, c
    ref = orc.backward(wl.scene, wl.cams, wl.tile, ob, dL.astype(np.float32).astype(np.float64),
                       fa)
    return {k: v.cpu().numpy() for k, v in g.items()}, ref


def test_backward_plain_matches_oracle(gs, orc):
    rng = np.random.default_rng(3003)
    sc = synth.blob_scene(rng, 3000, n_blobs=6, degree=3, log_scale=(-3.0, 0.5))
    cams = synth.orbit_cameras(rng, 2, 3.0, [(96, 80), (64, 64)])
    wl = synth.Workload("bwd", sc, cams, 16)
    g, ref = _run(gs, orc, wl)
    for k, rk in (("means", ref.means), ("scales", ref.scales), ("quats", ref.quats),
                  ("opac", ref.opac), ("sh", ref.sh)):
        _compare(k, g[k], rk, ref.mag[k])


@pytest.mark.parametrize("mv", [False, True])
def test_backward_foveated_matches_oracle(gs, orc, mv):
    rng = np.random.default_rng(4004)
    sc = synth.blob_scene(rng, 3000, n_blobs=6, degree=1, log_scale=(-3.0, 0.5))
    cams = synth.orbit_cameras(rng, 2, 3.0, [(96, 96), (80, 64)])
    m = synth.nested_levels(rng, sc.n, 4)
    f = synth.Foveation(4, m, synth.ring_tangents([5, 10, 16]), 6.0, synth.random_gaze(rng, cams))
    mvp = synth.multiversion_params(rng, sc, 4) if mv else None
    wl = synth.Workload("bwd_fov", sc, cams, 16, f)
    g, ref = _run(gs, orc, wl, fov=f, mv=mvp)
    for k, rk in (("means", ref.means), ("scales", ref.scales), ("quats", ref.quats),
                  ("opac", ref.opac), ("sh", ref.sh)):
        _compare(k, g[k], rk, ref.mag[k])
    if mv:
        _compare("opac_lv", g["opac_lv"], ref.opac_lv, ref.mag["opac_lv"])
        _compare("dc_lv", g["dc_lv"], ref.dc_lv, ref.mag["dc_lv"])


def test_backward_foveated_mixed_views_matches_oracle(gs, orc):
    # one foveated and one plain view in the same foveated call: the plain
    # view's pixels all composite level 1 with no band
    rng = np.random.default_rng(4005)
    sc = synth.blob_scene(rng, 3000, n_blobs=6, degree=1, log_scale=(-3.0, 0.5))
    cams = synth.orbit_cameras(rng, 2, 3.0, [(80, 96), (96, 72)])
    m = synth.nested_levels(rng, sc.n, 4)
    f = synth.Foveation(4, m, synth.ring_tangents([5, 10, 16]), 6.0, synth.random_gaze(rng, cams),
                        np.array([1, 0], np.uint8))
    wl = synth.Workload("bwd_fov_mixed", sc, cams, 16, f)
    g, ref = _run(gs, orc, wl, fov=f)
    for k, rk in (("means", ref.means), ("scales", ref.scales), ("quats", ref.quats),
                  ("opac", ref.opac), ("sh", ref.sh)):
        _compare(k, g[k], rk, ref.mag[k])


def test_autograd_l1_loss(gs, orc):
    import torch
    from paper_2407_00435_gb300 import autograd as ga
    wl = synth.workload(3, n=4000, views=2)
    sc = {k: v.clone().requires_grad_(True) for k, v in gs.scene_to_device(wl.scene).items()}
    r = gs.Renderer(wl.scene.n, wl.scene.sh_degree, wl.cams, backward=True)
    rng = np.random.default_rng(1003)
    target = torch.from_numpy(rng.uniform(0, 1, (r.P, 3)).astype(np.float32)).cuda()
    rgb = ga.render(sc, r)
    loss = ga.l1_loss(rgb, target)
    loss.backward()
    # oracle: dL/drgb of the mean absolute error, with the GPU's signs
    ob = orc.bin_pairs(wl.scene, wl.cams, wl.tile)
    img = orc.render(wl.scene, wl.cams, wl.tile, ob)
    dL = np.sign(rgb.detach().cpu().numpy() - target.cpu().numpy()).astype(np.float64) / rgb.numel()
    keep = (img.margin >= 1e-3) & (np.abs(img.rgb - target.cpu().numpy()).min(axis=1) > 1e-3)
    assert keep.mean() > 0.95
    # pixels dropped from the comparison are dropped on both sides
    ref = orc.backward(wl.scene, wl.cams, wl.tile, ob, dL * keep[:, None])
    g2 = {k: torch.empty_like(v) for k, v in sc.items()}
    out = r.alloc_outputs()
    r.project({k: v.detach() for k, v in sc.items()})
    r.bin_sort()
    r.render(out)
    r.backward(torch.from_numpy((dL * keep[:, None]).astype(np.float32)).cuda(), out, g2)
    for k, rk in (("means", ref.means), ("scales", ref.scales), ("opac", ref.opac),
                  ("sh", ref.sh)):
        _compare(k, g2[k].cpu().numpy(), rk, ref.mag[k])
    # autograd's gradient equals the C-ABI backward on the full loss
    dLfull = torch.from_numpy(dL.astype(np.float32)).cuda()
    r.backward(dLfull, out, g2)
    for k in sc:
        np.testing.assert_allclose(sc[k].grad.cpu().numpy(), g2[k].cpu().numpy(), rtol=1e-4,
                                   atol=1e-7)
