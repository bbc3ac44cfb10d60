"""The C-ABI library builds, loads and exports every entry point that
include/gs.h declares; host-side argument checks need no GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2407_00435_gb300 import build
    return C.CDLL(build.build())


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "gs_project" in names and "gs_render_backward" in names
    for n in names:
        assert hasattr(lib, n), n


def test_plan_init_validates_on_host(lib):
    from paper_2407_00435_gb300 import gs, synth
    cams = gs.cams_host(synth.camera_lookat((0, 0, -4), (0, 0, 0), 64, 48)[None])
    plan = C.create_string_buffer(int(lib.gs_plan_size()))
    lib.gs_plan_init.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p]
    assert lib.gs_plan_init(plan, 100, 4, cams, 1, None) == gs.GS_ERR_UNSUPPORTED
    assert lib.gs_plan_init(plan, -1, 0, cams, 1, None) == gs.GS_ERR_INVALID_ARG
    bad = gs.gs_config(12, 0, 0, 0, 0, 0)
    assert lib.gs_plan_init(plan, 100, 0, cams, 1, C.byref(bad)) == gs.GS_ERR_INVALID_ARG
    for cfg in (gs.gs_config(16, 0, 0, 0, 3, 0, 0),      # digit width below 4
                gs.gs_config(16, 0, 0, 0, 11, 0, 0),     # digit width above 10
                gs.gs_config(16, 32, 0, 0, 0, 0, 0),     # chunk below 64 points
                gs.gs_config(16, 256, 0, 0, 0, -1, 0)):  # negative chunk slots
        assert lib.gs_plan_init(plan, 100, 0, cams, 1, C.byref(cfg)) == gs.GS_ERR_INVALID_ARG
    # a separate model per level is a foveated plan
    mm = gs.gs_config(16, 0, gs.GS_FLAG_MULTI_MODEL, 0, 0, 0, 0)
    assert lib.gs_plan_init(plan, 100, 0, cams, 1, C.byref(mm)) == gs.GS_ERR_INVALID_ARG
    mm = gs.gs_config(16, 0, gs.GS_FLAG_MULTI_MODEL | gs.GS_FLAG_FOVEATED, 0, 0, 0, 0)
    assert lib.gs_plan_init(plan, 100, 0, cams, 1, C.byref(mm)) == gs.GS_OK
    lib.gs_workspace_size.argtypes = [C.c_void_p]
    lib.gs_workspace_size.restype = C.c_size_t
    # chunking reserves its slots; a plan without it does not
    assert lib.gs_plan_init(plan, 100, 0, cams, 1, C.byref(gs.gs_config(16, 256, 0, 0, 0, 0, 0))) == gs.GS_OK
    ws_chunked = lib.gs_workspace_size(plan)
    assert lib.gs_plan_init(plan, 100, 0, cams, 1, None) == gs.GS_OK
    assert lib.gs_workspace_size(plan) < ws_chunked
    lib.gs_plan_tiles.argtypes = [C.c_void_p]
    lib.gs_plan_tiles.restype = C.c_int64
    lib.gs_plan_pixels.argtypes = [C.c_void_p]
    lib.gs_plan_pixels.restype = C.c_int64
    assert lib.gs_plan_tiles(plan) == 4 * 3
    assert lib.gs_plan_pixels(plan) == 64 * 48
    lib.gs_workspace_size.argtypes = [C.c_void_p]
    lib.gs_workspace_size.restype = C.c_size_t
    assert lib.gs_workspace_size(plan) > 0
    # a null workspace is rejected before anything is enqueued
    lib.gs_bin_sort.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    assert lib.gs_bin_sort(plan, None, None) == gs.GS_ERR_INVALID_ARG
