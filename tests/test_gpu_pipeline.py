"""Pipelined frames from pinned host memory (HostFramePipeline): every
frame's image equals the image of the same scene rendered directly from
device memory (same kernels, same inputs: bit-exact), with frames of two
different scenes alternating so that a slot read before its upload landed,
or an image read before its render finished, would show."""
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


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_pipeline_frames_equal_direct_renders(gs, depth):
    import torch
    from paper_2407_00435_gb300.pipeline import HostFramePipeline
    rng = np.random.default_rng(808)
    scenes = [synth.blob_scene(rng, 40000, n_blobs=12, degree=2) for _ in range(2)]
    cams = synth.camera_lookat((0, 0, -4), (0, 0, 0), 320, 240)[None]
    r = gs.Renderer(scenes[0].n, 2, cams, tight=True)
    for sc in scenes:
        r.fit(gs.scene_to_device(sc), headroom=1.5)
    ref = []
    for sc in scenes:
        out = r.alloc_outputs()
        r.project(gs.scene_to_device(sc))
        r.bin_sort()
        r.render(out)
        ref.append(out["rgb"].cpu().numpy())
    hosts = [{k: torch.from_numpy(np.ascontiguousarray(getattr(sc, k))).pin_memory()
              for k in ("means", "scales", "quats", "opac", "sh")} for sc in scenes]
    n = 7
    rgb = [torch.zeros(r.P, 3).pin_memory() for _ in range(n)]
    pipe = HostFramePipeline(r, depth=depth)
    ea = torch.cuda.Event(enable_timing=True)
    eb = torch.cuda.Event(enable_timing=True)
    pipe.run([(hosts[i % 2], rgb[i]) for i in range(n)], ea, eb)
    torch.cuda.synchronize()
    assert ea.elapsed_time(eb) > 0
    code, c = r.counters()
    assert code == gs.GS_OK, c
    for i in range(n):
        np.testing.assert_array_equal(rgb[i].numpy(), ref[i % 2])


def test_pipeline_foveated_frames(gs):
    """The same with a foveated plan (two accumulators, band blending)."""
    import torch
    from paper_2407_00435_gb300.pipeline import HostFramePipeline
    rng = np.random.default_rng(809)
    sc = synth.blob_scene(rng, 30000, n_blobs=10, degree=1)
    cams = synth.camera_lookat((0, 0, -4), (0, 0, 0), 256, 192)[None]
    m = synth.nested_levels(rng, sc.n, 3)
    f = synth.Foveation(3, m, synth.ring_tangents([6.0, 12.0]), 8.0, synth.random_gaze(rng, cams))
    fd = gs.fov_to_device(f)
    r = gs.Renderer(sc.n, 1, cams, foveated=True)
    r.fit(gs.scene_to_device(sc), fd, headroom=1.5)
    out = r.alloc_outputs(fov=True)
    r.project(gs.scene_to_device(sc), fd)
    r.bin_sort()
    r.render(out, fov=True)
    ref = out["rgb"].cpu().numpy()
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(sc, k))).pin_memory()
            for k in ("means", "scales", "quats", "opac", "sh")}
    rgb = [torch.zeros(r.P, 3).pin_memory() for _ in range(3)]
    pipe = HostFramePipeline(r, fov=fd)
    pipe.run([(host, rgb[i]) for i in range(3)])
    torch.cuda.synchronize()
    for i in range(3):
        np.testing.assert_array_equal(rgb[i].numpy(), ref)
