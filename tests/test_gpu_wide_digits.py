"""Pair sorts with digits wider than 8 bits (9 or 10 bits: 512 or 1024 digit
values, one cooperative block per SM) against the FP64 oracle's FP32 binning:
sorted pairs and tile ranges bit-exact on many views whose tile ids need 18 or
19 bits, so that the balanced digit width really is 9 or 10."""
import numpy as np
import pytest

from paper_2407_00435_gb300 import synth
from test_gpu_forward import check_bins_exact, gpu_bins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_00435_gb300 import gs as _gs
    return _gs


@pytest.mark.parametrize("views,radix_bits,digit", [(16, 9, 9), (17, 10, 10)])
def test_wide_digit_pair_sort_bins_exact(gs, orc, views, radix_bits, digit):
    import torch
    rng = np.random.default_rng(5000 + views)
    sc = synth.blob_scene(rng, 8000, n_blobs=20, degree=1, log_scale=(-4.5, 0.5))
    cams = synth.orbit_cameras(rng, views, 3.0, [(1024, 1024)] * views)
    wl = synth.Workload("wide_digits", sc, cams, 8)
    tiles = views * (1024 // 8) ** 2
    tile_bits = int(tiles - 1).bit_length()
    passes = (tile_bits + radix_bits - 1) // radix_bits
    assert (tile_bits + passes - 1) // passes == digit     # the width the sort really uses
    r = gs.Renderer(sc.n, sc.sh_degree, cams, tile=8, radix_bits=radix_bits)
    dsc = gs.scene_to_device(sc)
    r.fit(dsc, None)
    torch.cuda.synchronize()
    gb = gpu_bins(gs, r)
    ob = orc.bin_pairs(sc, cams, 8, None)
    assert gb["K"] > 100000
    check_bins_exact(gb, ob, sc.n)
    # a second frame on the same plan gives the same pairs
    r.project(dsc, None)
    r.bin_sort()
    torch.cuda.synchronize()
    gb2 = gpu_bins(gs, r)
    np.testing.assert_array_equal(gb2["pair_tile"], gb["pair_tile"])
    np.testing.assert_array_equal(gb2["pair_item"], gb["pair_item"])
