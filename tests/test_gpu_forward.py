"""CUDA path vs the FP64 oracle: binning and sorting bit-exact, images
within 1e-3 max / 1e-5 mean absolute error, statistics and edge cases."""
import numpy as np
import pytest

from paper_2407_00435_gb300 import synth
from helpers import compare_images, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_00435_gb300 import gs as _gs
    return _gs


def gpu_bins(gs, r):
    """Visible items and sorted pairs read back from the workspace."""
    import torch
    code, c = r.counters()
    assert code == gs.GS_OK, c
    M, K = int(c["n_visible"]), int(c["n_pairs"])
    S = r.n * r.V                       # item slots j = i * V + v
    gid = r.region(gs.GS_REGION_ITEM_GID, torch.int32, S).cpu().numpy().astype(np.int64)
    view = r.region(gs.GS_REGION_ITEM_VIEW, torch.int32, S).cpu().numpy().astype(np.int64)
    depth = r.region(gs.GS_REGION_ITEM_DEPTH, torch.int32, S).cpu().numpy().view(np.uint32)
    count = r.region(gs.GS_REGION_ITEM_COUNT, torch.int32, S).cpu().numpy().view(np.uint32)
    vis = depth != 0xFFFFFFFF
    assert int(vis.sum()) == M
    j = np.arange(S)
    # a visible slot holds its own point and view
    np.testing.assert_array_equal(gid[vis], j[vis] // r.V)
    np.testing.assert_array_equal(view[vis], j[vis] % r.V)
    assert np.all(count[~vis] == 0)
    pt, pi = r.sorted_pairs(K)
    pt = pt.cpu().numpy().view(np.uint32).astype(np.uint64)
    pi = pi.cpu().numpy().astype(np.int64)
    ranges = r.region(gs.GS_REGION_RANGES, torch.int32, 2 * r.T_tiles).cpu().numpy().view(np.uint32).reshape(-1, 2)
    return dict(M=M, K=K, gid=gid, view=view, depth=depth, count=count, vis=vis, pair_tile=pt,
                pair_item=pi, ranges=ranges, nonfinite=int(c["n_nonfinite"]))


def check_bins_exact(gb, ob, n):
    # visible items: slot j = i * V + v on the GPU, v * n + i in the oracle
    V = len(gb["vis"]) // n if n else 1
    ov = (ob.vis == 1).reshape(V, n).T.reshape(-1)     # oracle visibility, slot order
    np.testing.assert_array_equal(gb["vis"], ov)
    assert gb["M"] == int(ov.sum())
    slots = np.nonzero(ov)[0]
    oracle_item = (slots % V) * n + slots // V
    np.testing.assert_array_equal(gb["depth"][slots], ob.dbits[oracle_item])
    np.testing.assert_array_equal(gb["count"][slots], ob.counts[oracle_item])
    # sorted pairs: key = tile << 32 | depth bits, value = v*n + i
    assert gb["K"] == ob.K
    j = gb["pair_item"]
    keys = (gb["pair_tile"] << np.uint64(32)) | gb["depth"][j].astype(np.uint64)
    np.testing.assert_array_equal(keys, ob.keys)
    np.testing.assert_array_equal(gb["view"][j] * n + gb["gid"][j], ob.vals.astype(np.int64))
    np.testing.assert_array_equal(gb["ranges"], ob.ranges)


def oracle_image(orc, wl, fov=None, mv=None, stats=False, bg=(0, 0, 0)):
    fa = orc.FovArrays.from_synth(fov, *(mv or (None, None))) if fov is not None else None
    ob = orc.bin_pairs(wl.scene, wl.cams, wl.tile, fa)
    img = orc.render(wl.scene, wl.cams, wl.tile, ob, fa, bg=bg, stats=stats)
    return ob, img, fa


def test_plain_128_n10k_bins_and_image(gs, orc):
    wl = synth.workload(0)
    r, out, _, _ = run_gpu(gs, wl, stats=True)
    ob, img, _ = oracle_image(orc, wl, stats=True)
    gb = gpu_bins(gs, r)
    check_bins_exact(gb, ob, wl.scene.n)
    rgb = out["rgb"].cpu().numpy()
    mx, mean, namb = compare_images(rgb, img)
    T = out["T"].cpu().numpy()
    amb = img.amb
    np.testing.assert_allclose(T[~amb], img.T[~amb, 0], atol=1e-5, rtol=1e-4)
    last = out["last"].cpu().numpy()
    assert np.array_equal(last[~amb], img.last[~amb, 0])
    st = out["stats"].cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(st[0], img.stats[0])           # tiles touched: exact
    # decision-based counts: equal up to the ambiguous pixels
    for k in (1, 2, 3):
        assert np.abs(st[k].astype(np.int64) - img.stats[k]).sum() <= 4 * (namb + 1)


def test_ragged_multiview_uneven_sizes(gs, orc):
    rng = np.random.default_rng(77)
    sc = synth.uniform_scene(rng, 3000, degree=2, log_scale=(-3.3, 0.6), dc_mode="coef")
    cams = synth.orbit_cameras(rng, 3, 4.0, [(100, 37), (64, 64), (131, 90)])
    wl = synth.Workload("ragged", sc, cams, 16)
    r, out, _, _ = run_gpu(gs, wl, bg=(0.1, 0.2, 0.3))
    ob, img, _ = oracle_image(orc, wl, bg=(0.1, 0.2, 0.3))
    check_bins_exact(gpu_bins(gs, r), ob, sc.n)
    compare_images(out["rgb"].cpu().numpy(), img)


@pytest.mark.parametrize("layout", ["wide", "ties"])
def test_depth_order_wide_range_and_ties(gs, orc, layout):
    """The depth sort ranks keys relative to the range of visible depths:
    a range wide enough that no digit is constant (depths 0.6 to 400), and a
    narrow one with many equal keys (two depth planes), whose ties must stay
    in point order.  Points behind the camera make invisible slots."""
    rng = np.random.default_rng(4242)
    n = 3000
    sc = synth.uniform_scene(rng, n, degree=1, log_scale=(-3.0, 0.5), dc_mode="coef")
    if layout == "wide":
        z = np.exp(rng.uniform(np.log(0.6), np.log(400.0), n)) - 4.0
    else:
        z = np.where(rng.random(n) < 0.5, 0.0, 0.5)
    z[rng.random(n) < 0.1] = -6.0          # behind the camera at z = -4
    sc.means[:, 2] = z.astype(np.float32)
    sc.means[:, :2] *= (0.5 * (z + 4.0)).clip(0.2, None)[:, None].astype(np.float32)
    cams = synth.camera_lookat((0, 0, -4), (0, 0, 0), 96, 80)[None]
    wl = synth.Workload("depth_" + layout, sc, cams, 16)
    r, out, _, _ = run_gpu(gs, wl)
    ob, img, _ = oracle_image(orc, wl)
    gb = gpu_bins(gs, r)
    assert 0 < gb["M"] < n
    check_bins_exact(gb, ob, n)
    compare_images(out["rgb"].cpu().numpy(), img)


def test_tile8(gs, orc):
    wl = synth.workload(0, n=4000)
    wl.tile = 8
    r, out, _, _ = run_gpu(gs, wl)
    ob, img, _ = oracle_image(orc, wl)
    check_bins_exact(gpu_bins(gs, r), ob, wl.scene.n)
    compare_images(out["rgb"].cpu().numpy(), img)


@pytest.mark.parametrize("mv", [False, True])
def test_foveated_multiview(gs, orc, mv):
    rng = np.random.default_rng(88)
    sc = synth.blob_scene(rng, 20000, n_blobs=20, degree=1)
    cams = synth.orbit_cameras(rng, 2, 3.0, [(160, 128), (96, 120)])
    m = synth.nested_levels(rng, sc.n, 4)
    gaze = synth.random_gaze(rng, cams)
    f = synth.Foveation(4, m, synth.ring_tangents([6, 12, 20]), 8.0, gaze,
                        np.array([1, 1], np.uint8))
    mvp = synth.multiversion_params(rng, sc, 4) if mv else None
    wl = synth.Workload("fov", sc, cams, 16, f)
    r, out, _, _ = run_gpu(gs, wl, fov=f, mv=mvp, stats=True)
    ob, img, _ = oracle_image(orc, wl, fov=f, mv=mvp, stats=True)
    check_bins_exact(gpu_bins(gs, r), ob, sc.n)
    tl = r.region(gs.GS_REGION_TILE_LEVEL, __import__("torch").uint8, r.T_tiles).cpu().numpy()
    np.testing.assert_array_equal(tl, ob.tile_level)
    compare_images(out["rgb"].cpu().numpy(), img)
    T = out["T"].cpu().numpy().reshape(-1, 2)
    amb = img.amb
    np.testing.assert_allclose(T[~amb], img.T[~amb], atol=1e-5, rtol=1e-4)


def test_mixed_plain_and_foveated_views(gs, orc):
    rng = np.random.default_rng(99)
    sc = synth.blob_scene(rng, 15000, n_blobs=15, degree=0)
    cams = synth.orbit_cameras(rng, 3, 3.5, [(128, 128), (80, 64), (144, 96)])
    m = synth.nested_levels(rng, sc.n, 3)
    f = synth.Foveation(3, m, synth.ring_tangents([8, 16]), 6.0, synth.random_gaze(rng, cams),
                        np.array([1, 0, 1], np.uint8))
    wl = synth.Workload("mixed", sc, cams, 16, f)
    r, out, _, _ = run_gpu(gs, wl, fov=f)
    ob, img, _ = oracle_image(orc, wl, fov=f)
    check_bins_exact(gpu_bins(gs, r), ob, sc.n)
    compare_images(out["rgb"].cpu().numpy(), img)


def test_empty_scene_and_empty_view(gs, orc):
    import torch
    # no points at all: background everywhere
    sc = synth.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32),
                     np.zeros((0, 4), np.float32), np.zeros(0, np.float32),
                     np.zeros((0, 1, 3), np.float32), 0)
    cams = synth.camera_lookat((0, 0, -4), (0, 0, 0), 40, 24)[None]
    wl = synth.Workload("empty", sc, cams, 16)
    r = gs.Renderer(0, 0, cams)
    z = {k: torch.zeros(1, device="cuda") for k in ("means", "scales", "quats", "opac", "sh")}
    r.project(z)
    r.bin_sort()
    out = r.alloc_outputs()
    r.render(out, bg=(0.25, 0.5, 0.75))
    code, c = r.counters()
    assert code == gs.GS_OK and c["n_visible"] == 0 and c["n_pairs"] == 0
    np.testing.assert_allclose(out["rgb"].cpu().numpy(), np.tile([0.25, 0.5, 0.75], (40 * 24, 1)))
    assert np.all(out["T"].cpu().numpy() == 1.0) and np.all(out["last"].cpu().numpy() == -1)
    # a scene entirely behind the camera
    sc2 = synth.uniform_scene(np.random.default_rng(1), 500)
    sc2.means[:, 2] = -10.0
    wl2 = synth.Workload("behind", sc2, cams, 16)
    r2, out2, _, _ = run_gpu(gs, wl2)
    assert r2.counters()[1]["n_visible"] == 0
    assert np.all(out2["rgb"].cpu().numpy() == 0.0)


def test_nonfinite_points_are_culled_and_counted(gs, orc):
    wl = synth.workload(0, n=2000)
    wl.scene.means[5, 0] = np.nan
    wl.scene.scales[7, 1] = np.inf
    wl.scene.sh[9, 0, 2] = np.nan
    r, out, _, _ = run_gpu(gs, wl)
    gb = gpu_bins(gs, r)
    assert gb["nonfinite"] == 3
    ob, img, _ = oracle_image(orc, wl)
    check_bins_exact(gb, ob, wl.scene.n)
    assert np.isfinite(out["rgb"].cpu().numpy()).all()
    compare_images(out["rgb"].cpu().numpy(), img)


def test_pair_capacity_overflow_is_reported(gs):
    wl = synth.workload(0, n=3000)
    r, out, _, _ = run_gpu(gs, wl, max_pairs=100)
    code, c = r.counters()
    assert code == gs.GS_ERR_CAPACITY
    assert c["n_pairs"] > 100
    assert np.isfinite(out["rgb"].cpu().numpy()).all()
    r.clear_error()
    assert r.counters()[0] == gs.GS_OK


def test_full_size_1080p_n1M_bins_exact_and_sampled_pixels(gs, orc):
    wl = synth.workload(1)
    r, out, _, _ = run_gpu(gs, wl)
    ob = orc.bin_pairs(wl.scene, wl.cams, wl.tile)
    check_bins_exact(gpu_bins(gs, r), ob, wl.scene.n)
    rng = np.random.default_rng(5)
    P = 1920 * 1080
    lens = (ob.ranges[:, 1] - ob.ranges[:, 0]).astype(np.int64)
    # sample pixels: uniform plus the heaviest tiles and the ragged last row
    heavy = np.argsort(lens)[-4:]
    pix = list(rng.choice(P, 3000, replace=False))
    for t in heavy:
        ty, tx = divmod(int(t), 120)
        for k in range(0, 256, 9):
            x, y = tx * 16 + k % 16, ty * 16 + k // 16
            if y < 1080:
                pix.append(y * 1920 + x)
    pix += [1079 * 1920 + x for x in range(0, 1920, 37)]
    pix = np.array(sorted(set(pix)), np.int64)
    img = orc.render(wl.scene, wl.cams, 16, ob, pix=pix)
    rgb = out["rgb"].cpu().numpy()[pix]
    compare_images(rgb, img)
