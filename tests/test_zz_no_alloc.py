"""The allocation-free pair sort (gs_sort_pairs_static) against the pair
sort inside gs_bin_sort.

gs_sort_pairs_static exists for callers that cannot allocate device memory
(a pool that must not grow, a host application that forbids cudaMalloc after
start-up, a real-time path where an allocation could block): it sorts the
caller's buffers with a static scratch array of the library.  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes as C

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


def _reference_pairs(gs, wl):
    """Sorted pairs from gs_bin_sort, and the same pairs in the order the
    binning emits them (items in depth order, each item's tiles row-major)."""
    import torch
    sc = gs.scene_to_device(wl.scene)
    r = gs.Renderer(wl.scene.n, wl.scene.sh_degree, wl.cams)
    c = r.fit(sc)
    K = int(c["n_pairs"])
    pt, pi = r.sorted_pairs(K)
    tile = pt.cpu().numpy().view(np.uint32)
    item = pi.cpu().numpy().view(np.uint32)
    depth = r.region(gs.GS_REGION_ITEM_DEPTH, torch.int32, r.n * r.V).cpu().numpy().view(np.uint32)
    emit = np.lexsort((tile, item, depth[item]))
    bits = max(1, int(r.T_tiles - 1).bit_length())
    return tile, item, tile[emit].copy(), item[emit].copy(), bits


def _static_sort(gs, keys, vals, bits):
    import torch
    n = len(keys)
    kin = torch.from_numpy(keys.view(np.int32)).cuda()
    vin = torch.from_numpy(vals.view(np.int32)).cuda()
    kout = torch.full_like(kin, -1)
    vout = torch.full_like(vin, -1)
    s = torch.cuda.current_stream().cuda_stream
    code = gs.lib().gs_sort_pairs_static(kin.data_ptr(), vin.data_ptr(), n, bits,
                                         kout.data_ptr(), vout.data_ptr(), s)
    assert code == gs.GS_OK
    st = C.c_uint32(99)
    assert gs.lib().gs_sort_pairs_static_status(C.byref(st), s) == gs.GS_OK
    assert st.value == gs.GS_OK
    return kout.cpu().numpy().view(np.uint32), vout.cpu().numpy().view(np.uint32)


def test_static_sort_matches_bin_sort_two_calls_in_a_row(gs):
    # two different workloads back to back: the second call must not see
    # anything left in the shared scratch by the first
    for wl in (synth.workload(0), synth.workload(3, n=20000, views=2)):
        tile, item, k_in, v_in, bits = _reference_pairs(gs, wl)
        assert len(tile) <= (1 << 20)
        k_out, v_out = _static_sort(gs, k_in, v_in, bits)
        np.testing.assert_array_equal(k_out, tile)
        np.testing.assert_array_equal(v_out, item)


def test_static_sort_rejects_oversize_and_overlap(gs):
    import torch
    lib = gs.lib()
    buf = torch.zeros(8, dtype=torch.int32, device="cuda")
    p = buf.data_ptr()
    s = torch.cuda.current_stream().cuda_stream
    assert lib.gs_sort_pairs_static(p, p + 16, (1 << 20) + 1, 8, p, p, s) == gs.GS_ERR_INVALID_ARG
    assert lib.gs_sort_pairs_static(p, p + 16, 4, 8, p, p + 16, s) == gs.GS_ERR_INVALID_ARG
    assert lib.gs_sort_pairs_static(p, p + 16, 4, 0, p, p, s) == gs.GS_ERR_INVALID_ARG


@pytest.mark.parametrize("bits,n", [(5, 70001), (13, 1 << 20), (20, 333333), (32, 123457)])
def test_static_sort_random_keys_against_numpy(gs, bits, n):
    # key widths of one to four passes (20 bits: three passes, the odd count
    # that routes the result through the static scratch), the size limit,
    # ragged sizes and inputs that start 4 bytes past a 16-byte boundary
    # (the plain-load path of the sort's partition staging)
    import torch
    rng = np.random.default_rng(bits * 1000 + n % 997)
    keys = rng.integers(0, 1 << bits, n, dtype=np.uint64).astype(np.uint32)
    keys[: n // 7] = keys[n // 3]                  # a long run of equal keys
    vals = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    order = np.argsort(keys, kind="stable")
    s = torch.cuda.current_stream().cuda_stream
    for offset in (0, 1):                          # in int32 elements
        kin = torch.empty(n + 4, dtype=torch.int32, device="cuda")
        vin = torch.empty(n + 4, dtype=torch.int32, device="cuda")
        kin[offset:offset + n] = torch.from_numpy(keys.view(np.int32)).cuda()
        vin[offset:offset + n] = torch.from_numpy(vals.view(np.int32)).cuda()
        kout = torch.full((n + 4,), -1, dtype=torch.int32, device="cuda")
        vout = torch.full((n + 4,), -1, dtype=torch.int32, device="cuda")
        ptr = lambda t: t.data_ptr() + 4 * offset
        code = gs.lib().gs_sort_pairs_static(ptr(kin), ptr(vin), n, bits, ptr(kout), ptr(vout), s)
        assert code == gs.GS_OK
        st = C.c_uint32(99)
        assert gs.lib().gs_sort_pairs_static_status(C.byref(st), s) == gs.GS_OK
        ko = kout.cpu().numpy().view(np.uint32)
        vo = vout.cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(ko[offset:offset + n], keys[order])
        np.testing.assert_array_equal(vo[offset:offset + n], vals[order])
        # nothing written outside the n outputs
        assert np.all(ko[:offset] == 0xffffffff) and np.all(ko[offset + n:] == 0xffffffff)
