"""Failure detection on the GPU without a GPU fault: a bounded device-side
wait that runs out reports GS_ERR_TIMEOUT through the status word, the
kernel returns, and the context stays usable for the next frame.

The projection's bulk-copy waits take their poll limit from the plan
(gs_config.wait_spins); a negative limit makes every wait give up at once,
as a wait on a copy that never lands would after its full limit.  The copies
that were issued still land before the blocks leave (that drain keeps the
full limit), so nothing is left in flight."""
import numpy as np
import pytest

from paper_2407_00435_gb300 import synth
from helpers import compare_images

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_00435_gb300 import gs as _gs
    return _gs


def test_projection_wait_that_runs_out_reports_timeout_and_the_next_frame_renders(gs, orc):
    import torch
    wl = synth.workload(0, n=4096)       # 32 full blocks of 128 points take the bulk-copy path
    sc = gs.scene_to_device(wl.scene)
    bad = gs.Renderer(wl.scene.n, wl.scene.sh_degree, wl.cams, wait_spins=-1)
    bad.project(sc)
    code, c = bad.counters()
    assert code == gs.GS_ERR_TIMEOUT, (code, c)
    # the status word is sticky for the frame and reset by the next projection
    code2, _ = bad.counters()
    assert code2 == gs.GS_ERR_TIMEOUT
    # the same device and scene, default waits: a correct frame
    good = gs.Renderer(wl.scene.n, wl.scene.sh_degree, wl.cams)
    good.fit(sc)
    out = good.alloc_outputs()
    good.render(out)
    torch.cuda.synchronize()
    code3, c3 = good.counters()
    assert code3 == gs.GS_OK, c3
    ob = orc.bin_pairs(wl.scene, wl.cams, wl.tile)
    assert int(c3["n_pairs"]) == ob.K
    compare_images(out["rgb"].cpu().numpy(), orc.render(wl.scene, wl.cams, wl.tile, ob),
                   label="after a timeout")
    # and the failing plan itself recovers once re-planned with default waits
    again = gs.Renderer(wl.scene.n, wl.scene.sh_degree, wl.cams)
    again.project(sc)
    assert again.counters()[0] == gs.GS_OK


def test_positive_poll_limit_behaves_like_the_default(gs):
    wl = synth.workload(0, n=4096)
    sc = gs.scene_to_device(wl.scene)
    r = gs.Renderer(wl.scene.n, wl.scene.sh_degree, wl.cams, wait_spins=1 << 16)
    r.fit(sc)
    assert r.counters()[0] == gs.GS_OK
