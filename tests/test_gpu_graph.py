"""A whole frame (projection, pair count on the library's side stream,
binning, render) captured into one CUDA graph and replayed gives the image
of the same frame launched directly (same kernels, same inputs: bit-exact),
also after the scene changes in place between replays."""
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


@pytest.mark.parametrize("foveated", [False, True])
def test_graph_replay_equals_direct_frame(gs, foveated):
    import torch
    rng = np.random.default_rng(1212)
    scenes = [synth.blob_scene(rng, 20000, n_blobs=8, degree=1) for _ in range(2)]
    cams = synth.orbit_cameras(rng, 2, 3.5, [(160, 120), (96, 128)])
    f = None
    if foveated:
        m = synth.nested_levels(rng, scenes[0].n, 3)
        f = gs.fov_to_device(synth.Foveation(3, m, synth.ring_tangents([6.0, 12.0]), 6.0,
                                             synth.random_gaze(rng, cams)))
    sc = gs.scene_to_device(scenes[0])
    r = gs.Renderer(scenes[0].n, 1, cams, foveated=foveated, tight=True)
    for s_ in scenes:
        r.fit(gs.scene_to_device(s_), f, headroom=1.5)
    out = r.alloc_outputs(fov=foveated)

    def frame():
        r.project(sc, f)
        r.bin_sort()
        r.render(out, fov=foveated)

    refs = []
    for s_ in scenes:
        for k in sc:
            sc[k].copy_(gs.scene_to_device(s_)[k])
        frame()
        torch.cuda.synchronize()
        refs.append(out["rgb"].cpu().numpy())
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        frame()
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=st):
            frame()
    torch.cuda.current_stream().wait_stream(st)
    for i in range(4):
        for k in sc:
            sc[k].copy_(gs.scene_to_device(scenes[i % 2])[k])
        out["rgb"].zero_()
        graph.replay()
        torch.cuda.synchronize()
        code, c = r.counters()
        assert code == gs.GS_OK, c
        np.testing.assert_array_equal(out["rgb"].cpu().numpy(), refs[i % 2])
