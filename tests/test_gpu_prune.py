"""Efficiency-aware pruning and scale decay on the GPU (Sec. 3.2-3.4) against
the FP64 reference in oracle/prune.py."""
import numpy as np
import pytest

from paper_2407_00435_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_00435_gb300 import gs as _gs
    return _gs


def _pose_stats(gs, sc_d, scene, cam):
    r = gs.Renderer(scene.n, scene.sh_degree, cam[None], tight=True)
    r.fit(sc_d)
    out = r.alloc_outputs(stats=True)
    r.render(out)
    assert r.counters()[0] == gs.GS_OK
    return out["stats"]


def test_ce_max_over_poses(gs):
    import torch
    from oracle import prune as P
    rng = np.random.default_rng(71)
    sc = synth.blob_scene(rng, 8000, n_blobs=10, degree=1)
    cams = synth.orbit_cameras(rng, 3, 3.0, [(128, 96)] * 3)
    d = gs.scene_to_device(sc)
    ce = torch.zeros(sc.n, device="cuda")
    stats = []
    for cam in cams:
        st = _pose_stats(gs, d, sc, cam)
        gs.gs_ce_update(sc.n, st, ce)
        stats.append(st.cpu().numpy().view(np.uint32).reshape(4, sc.n))
    got = ce.cpu().numpy()
    # the same FP32 divisions and maxima on the host: bit-exact
    ref32 = np.zeros(sc.n, np.float32)
    for st in stats:
        c = st[0] > 0
        q = np.zeros(sc.n, np.float32)
        q[c] = st[3][c].astype(np.float32) / st[0][c].astype(np.float32)
        ref32 = np.where(c, np.maximum(ref32, q), ref32)
    np.testing.assert_array_equal(got, ref32)
    np.testing.assert_allclose(got, P.ce_max(stats), rtol=1e-7, atol=0)
    assert (got > 0).sum() > 1000


@pytest.mark.parametrize("n", [1, 4096, 200003])
def test_prune_mask_matches_reference(gs, n):
    import torch
    from oracle import prune as P
    rng = np.random.default_rng(72 + n)
    ce = (rng.integers(0, 64, n) / 16.0).astype(np.float32)     # many exact ties
    cams = synth.camera_lookat((0, 0, -4), (0, 0, 0), 32, 32)[None]
    r = gs.Renderer(n, 0, cams)
    for fraction in (0.1, 0.0, 0.5, 1.0):
        keep = r.prune_mask(torch.from_numpy(ce).cuda(), fraction).cpu().numpy().astype(bool)
        np.testing.assert_array_equal(keep, P.prune_keep(ce.astype(np.float64), fraction))


def test_compact_points_is_stable(gs):
    import torch
    rng = np.random.default_rng(73)
    sc = synth.uniform_scene(rng, 30001, degree=2)
    d = gs.scene_to_device(sc)
    r = gs.Renderer(sc.n, 2, synth.camera_lookat((0, 0, -4), (0, 0, 0), 32, 32)[None])
    keep_np = rng.uniform(size=sc.n) < 0.7
    out = r.compact(d, torch.from_numpy(keep_np.astype(np.uint8)).cuda())
    assert out["means"].shape[0] == keep_np.sum()
    for k, arr in (("means", sc.means), ("scales", sc.scales), ("quats", sc.quats),
                   ("opac", sc.opac), ("sh", sc.sh)):
        np.testing.assert_array_equal(out[k].cpu().numpy(), arr[keep_np])


def test_weighted_scale_and_gradient(gs):
    import torch
    from oracle import prune as P
    rng = np.random.default_rng(74)
    n = 100003
    scales = np.exp(rng.normal(-3, 0.8, (n, 3))).astype(np.float32)
    stats = np.zeros((4, n), np.uint32)
    stats[1] = rng.integers(0, 60, n)
    T, gamma = 12.0, 0.25
    ws_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    g_d = torch.zeros((n, 3), device="cuda")
    gs.gs_weighted_scale(n, torch.from_numpy(scales).cuda(),
                         torch.from_numpy(stats.view(np.int32)).cuda(), T, gamma, ws_d, g_d)
    ws, g = P.weighted_scale(scales.astype(np.float64), stats[1], T)
    assert float(ws_d.item()) == pytest.approx(ws, rel=1e-6)
    np.testing.assert_allclose(g_d.cpu().numpy(), gamma * g, rtol=1e-6, atol=1e-12)


def test_pruning_round_renders_the_pruned_scene(gs, orc):
    import torch
    from helpers import compare_images
    rng = np.random.default_rng(75)
    sc = synth.blob_scene(rng, 6000, n_blobs=8, degree=1)
    cams = synth.orbit_cameras(rng, 2, 3.0, [(96, 80)] * 2)
    d = gs.scene_to_device(sc)
    ce = torch.zeros(sc.n, device="cuda")
    for cam in cams:
        gs.gs_ce_update(sc.n, _pose_stats(gs, d, sc, cam), ce)
    r = gs.Renderer(sc.n, 1, cams, tight=True)
    keep = r.prune_mask(ce, 0.1)
    pruned = r.compact(d, keep)
    keep_np = keep.cpu().numpy().astype(bool)
    assert pruned["means"].shape[0] == sc.n - int(0.1 * sc.n)
    sp = synth.Scene(sc.means[keep_np], sc.scales[keep_np], sc.quats[keep_np], sc.opac[keep_np],
                     sc.sh[keep_np], 1)
    rp = gs.Renderer(sp.n, 1, cams, tight=True)
    rp.fit({k: v.contiguous() for k, v in pruned.items()})
    out = rp.alloc_outputs()
    rp.render(out)
    ob = orc.bin_pairs(sp, cams, 16, tight=True)
    compare_images(out["rgb"].cpu().numpy(), orc.render(sp, cams, 16, ob))


def test_scale_decay_autograd(gs):
    import torch
    from oracle import prune as P
    from paper_2407_00435_gb300 import autograd as ga
    rng = np.random.default_rng(76)
    n = 5000
    s_np = np.exp(rng.normal(-2, 0.7, (n, 3))).astype(np.float32)
    stats = np.zeros((4, n), np.uint32)
    stats[1] = rng.integers(0, 40, n)
    s = torch.from_numpy(s_np).cuda().requires_grad_(True)
    loss = ga.scale_decay(s, torch.from_numpy(stats.view(np.int32)).cuda(), 10.0, 0.5)
    loss.backward()
    ws, g = P.weighted_scale(s_np.astype(np.float64), stats[1], 10.0)
    assert float(loss.item()) == pytest.approx(0.5 * ws, rel=1e-6)
    np.testing.assert_allclose(s.grad.cpu().numpy(), 0.5 * g, rtol=1e-6, atol=1e-12)
