"""Heavy-tile chunking of the render (persistent work queue, (C, T) merge in
list order, re-walk of the chunk holding the early stop) against the FP64
oracle and against whole-tile rendering of the same plan inputs."""
import numpy as np
import pytest

from paper_2407_00435_gb300 import synth
from helpers import compare_grads, compare_images, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_00435_gb300 import gs as _gs
    return _gs


def _oracle(orc, wl, fov=None, mv=None, bg=(0, 0, 0)):
    fa = orc.FovArrays.from_synth(fov, *(mv or (None, None))) if fov is not None else None
    ob = orc.bin_pairs(wl.scene, wl.cams, wl.tile, fa)
    return ob, orc.render(wl.scene, wl.cams, wl.tile, ob, fa, bg=bg), fa


def _dense_scene(seed, n, views, degree=1):
    """Blobs of opaque points: long tile lists in which most pixels stop."""
    rng = np.random.default_rng(seed)
    sc = synth.blob_scene(rng, n, n_blobs=8, degree=degree, log_scale=(-3.0, 0.4))
    sc.opac[:] = np.clip(sc.opac * 1.5, 0.05, 0.98).astype(np.float32)
    cams = synth.orbit_cameras(rng, len(views), 3.0, views)
    return synth.Workload("dense", sc, cams, 16)


@pytest.mark.parametrize("chunk", [64, 200])
def test_chunked_plain_matches_oracle_and_whole_tiles(gs, orc, chunk):
    wl = _dense_scene(5005, 12000, [(96, 80), (64, 48)])
    rc, outc, _, _ = run_gpu(gs, wl, chunk=chunk, bg=(0.2, 0.1, 0.0))
    code, c = rc.counters()
    assert code == gs.GS_OK, c
    rw, outw, _, _ = run_gpu(gs, wl, bg=(0.2, 0.1, 0.0))
    ob, img, _ = _oracle(orc, wl, bg=(0.2, 0.1, 0.0))
    lens = ob.ranges[:, 1] - ob.ranges[:, 0]
    assert (lens > chunk).mean() > 0.3          # most tiles are split
    compare_images(outc["rgb"].cpu().numpy(), img)
    amb = img.amb
    T = outc["T"].cpu().numpy()
    last = outc["last"].cpu().numpy()
    np.testing.assert_allclose(T[~amb], img.T[~amb, 0], atol=1e-5, rtol=1e-4)
    np.testing.assert_array_equal(last[~amb], img.last[~amb, 0])
    # pixels that stop inside a later chunk exercise the merge's re-walk
    stopped_late = (~amb) & (img.T[:, 0] < 0.0102) & (img.last[:, 0] >= chunk)
    assert stopped_late.sum() > 50
    # chunked vs whole tiles: the same decisions, colours equal to rounding
    dw = np.abs(outc["rgb"].cpu().numpy() - outw["rgb"].cpu().numpy()).max(axis=1)
    assert dw[~amb].max() <= 1e-5
    np.testing.assert_array_equal(last[~amb], outw["last"].cpu().numpy()[~amb])


@pytest.mark.parametrize("mv", [False, True])
def test_chunked_foveated_matches_oracle(gs, orc, mv):
    wl = _dense_scene(6006, 15000, [(128, 112), (80, 96)])
    rng = np.random.default_rng(6007)
    m = synth.nested_levels(rng, wl.scene.n, 4)
    f = synth.Foveation(4, m, synth.ring_tangents([5, 10, 16]), 8.0,
                        synth.random_gaze(rng, wl.cams))
    mvp = synth.multiversion_params(rng, wl.scene, 4) if mv else None
    wl = synth.Workload("dense_fov", wl.scene, wl.cams, 16, f)
    r, out, _, _ = run_gpu(gs, wl, fov=f, mv=mvp, chunk=96)
    assert r.counters()[0] == gs.GS_OK
    ob, img, _ = _oracle(orc, wl, fov=f, mv=mvp)
    assert ((ob.ranges[:, 1] - ob.ranges[:, 0]) > 96).mean() > 0.2
    compare_images(out["rgb"].cpu().numpy(), img)
    T = out["T"].cpu().numpy().reshape(-1, 2)
    last = out["last"].cpu().numpy().reshape(-1, 2)
    amb = img.amb
    np.testing.assert_allclose(T[~amb], img.T[~amb], atol=1e-5, rtol=1e-4)
    np.testing.assert_array_equal(last[~amb], img.last[~amb])


def test_chunk_slot_overflow_renders_whole_tiles(gs, orc):
    # 16 tiles of ~1000+ pairs with chunk 64 ask for far more slots than the
    # 40 the plan is given: the tiles that do not fit render whole
    wl = _dense_scene(7007, 20000, [(64, 64)])
    r, out, _, _ = run_gpu(gs, wl, chunk=64, chunk_slots=40)
    code, c = r.counters()
    assert code == gs.GS_OK, c
    ob, img, _ = _oracle(orc, wl)
    lens = ob.ranges[:, 1] - ob.ranges[:, 0]
    need = np.ceil(lens[lens > 64] / 64)
    assert need.sum() > 40 and need.min() <= 40    # some tiles fit, the others do not
    compare_images(out["rgb"].cpu().numpy(), img)


def test_chunked_tile8_and_ragged(gs, orc):
    wl = _dense_scene(8008, 6000, [(70, 45), (33, 61)])
    wl.tile = 8
    r, out, _, _ = run_gpu(gs, wl, chunk=64)
    assert r.counters()[0] == gs.GS_OK
    ob, img, _ = _oracle(orc, wl)
    compare_images(out["rgb"].cpu().numpy(), img)


def test_backward_after_chunked_forward(gs, orc):
    import torch
    wl = _dense_scene(9009, 3000, [(80, 64)], degree=2)
    sc = gs.scene_to_device(wl.scene)
    r = gs.Renderer(wl.scene.n, wl.scene.sh_degree, wl.cams, backward=True, chunk=64)
    r.fit(sc)
    out = r.alloc_outputs()
    r.render(out)
    ob, img, _ = _oracle(orc, wl)
    rng = np.random.default_rng(9010)
    dL = rng.uniform(-1, 1, (r.P, 3))
    dL[img.margin < 1e-3] = 0.0
    S = (wl.scene.sh_degree + 1) ** 2
    g = {k: torch.empty(s, device="cuda") for k, s in
         (("means", (wl.scene.n, 3)), ("scales", (wl.scene.n, 3)), ("quats", (wl.scene.n, 4)),
          ("opac", (wl.scene.n,)), ("sh", (wl.scene.n, S, 3)))}
    r.backward(torch.from_numpy(dL.astype(np.float32)).cuda(), out, g)
    assert r.counters()[0] == gs.GS_OK
    ref = orc.backward(wl.scene, wl.cams, wl.tile, ob, dL.astype(np.float32).astype(np.float64))
    for k, rk in (("means", ref.means), ("scales", ref.scales), ("quats", ref.quats),
                  ("opac", ref.opac), ("sh", ref.sh)):
        compare_grads(k, g[k].cpu().numpy(), rk, ref.mag[k])


def test_autotuner_picks_a_candidate_and_its_image_matches(gs, orc, tmp_path):
    from paper_2407_00435_gb300.autotune import autotune
    wl = _dense_scene(1111, 8000, [(96, 96)])
    sc = gs.scene_to_device(wl.scene)
    cands = [{"tile": 16, "radix_bits": 0, "chunk": 0}, {"tile": 16, "radix_bits": 0, "chunk": 128},
             {"tile": 8, "radix_bits": 6, "chunk": 64}]
    cache = str(tmp_path / "tune.json")
    res = autotune(sc, wl.scene.n, wl.scene.sh_degree, wl.cams, candidates=cands, frames=2,
                   cache_path=cache)
    assert res["options"] in [{k: c[k] for k in ("tile", "radix_bits", "chunk")} for c in cands]
    assert all(t["ms"] is not None for t in res["trials"])
    assert autotune(sc, wl.scene.n, wl.scene.sh_degree, wl.cams, candidates=cands,
                    cache_path=cache) == res          # served from the cache
    opt = res["options"]
    wl.tile = opt["tile"]
    r, out, _, _ = run_gpu(gs, wl, chunk=opt["chunk"])
    ob, img, _ = _oracle(orc, wl)
    compare_images(out["rgb"].cpu().numpy(), img)
