"""Thin ctypes binding of ``libgs.so`` (the C ABI in ``include/gs.h``).

Argument marshalling only: every stage runs in the library's CUDA kernels.
PyTorch provides device memory and streams.  There is no CPU fallback: if
the library is missing or fails to load, importing the binding raises.

Function names follow the C ABI (``gs_project``, ``gs_bin_sort``,
``gs_render``, ``gs_render_fov``, ``gs_render_backward``, ...).  The
:class:`Renderer` class owns a plan and a workspace and is what the tests,
the benchmark and the autograd wrapper use.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

GS_OK, GS_ERR_INVALID_ARG, GS_ERR_CAPACITY, GS_ERR_TIMEOUT, GS_ERR_CUDA, GS_ERR_UNSUPPORTED = range(6)
GS_FLAG_FOVEATED = 1
GS_FLAG_BACKWARD = 2
GS_FLAG_TIGHT = 4
GS_FLAG_MULTI_MODEL = 8
GS_MAX_LEVELS = 8
(GS_REGION_ITEM_GID, GS_REGION_ITEM_VIEW, GS_REGION_ITEM_DEPTH, GS_REGION_ITEM_COUNT) = (1, 2, 3, 4)
GS_REGION_RANGES, GS_REGION_TILE_LEVEL = 7, 8

_STATUS_NAMES = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_CAPACITY",
                 3: "GS_ERR_TIMEOUT", 4: "GS_ERR_CUDA", 5: "GS_ERR_UNSUPPORTED"}


class GsError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {_STATUS_NAMES.get(code, code)}")
        self.code = code


class gs_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float),
                ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32), ("znear", C.c_float),
                ("zfar", C.c_float)]


class gs_scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("reserved", C.c_int32),
                ("means", C.c_void_p), ("scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacities", C.c_void_p), ("sh", C.c_void_p)]


class gs_fov(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("band_px", C.c_float),
                ("ring_tan", C.c_float * (GS_MAX_LEVELS - 1)), ("bound_m", C.c_void_p),
                ("gaze_px", C.c_void_p), ("view_fov", C.c_void_p), ("opacity_lv", C.c_void_p),
                ("dc_lv", C.c_void_p)]


class gs_config(C.Structure):
    _fields_ = [("tile", C.c_int32), ("chunk", C.c_int32), ("flags", C.c_int32),
                ("max_levels", C.c_int32), ("radix_bits", C.c_int32), ("chunk_slots", C.c_int32),
                ("max_pairs", C.c_int64), ("wait_spins", C.c_int32), ("reserved", C.c_int32)]


class gs_counters(C.Structure):
    _fields_ = [("status", C.c_uint32), ("reserved", C.c_uint32), ("n_visible", C.c_uint64),
                ("n_pairs", C.c_uint64), ("n_nonfinite", C.c_uint64),
                ("n_evals", C.c_uint64), ("n_blends", C.c_uint64)]


assert C.sizeof(gs_camera) == 80


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        path = _build.build()
    lib = C.CDLL(path)
    p, s = C.c_void_p, C.c_int32
    lib.gs_plan_size.restype = C.c_size_t
    lib.gs_plan_init.argtypes = [p, C.c_int64, s, p, s, p]
    lib.gs_plan_init.restype = s
    lib.gs_workspace_size.argtypes = [p]
    lib.gs_workspace_size.restype = C.c_size_t
    lib.gs_project.argtypes = [p, p, C.c_size_t, p, p, p, p]
    lib.gs_project.restype = s
    lib.gs_bin_sort.argtypes = [p, p, p]
    lib.gs_bin_sort.restype = s
    lib.gs_render.argtypes = [p, p, p, p, p, p, p, p]
    lib.gs_render.restype = s
    lib.gs_render_fov.argtypes = [p, p, p, p, p, p, p, p]
    lib.gs_render_fov.restype = s
    lib.gs_render_backward.argtypes = [p, p, p, p, p, p, p, p, p, p, p, p, p, p]
    lib.gs_render_backward.restype = s
    lib.gs_get_error.argtypes = [p, p, p, p]
    lib.gs_get_error.restype = s
    lib.gs_clear_error.argtypes = [p, p, p]
    lib.gs_clear_error.restype = s
    lib.gs_ws_region.argtypes = [p, s, p, p]
    lib.gs_ws_region.restype = s
    lib.gs_sorted_pairs.argtypes = [p, p, p, p, p]
    lib.gs_sorted_pairs.restype = s
    lib.gs_plan_tiles.argtypes = [p]
    lib.gs_plan_tiles.restype = C.c_int64
    lib.gs_plan_pixels.argtypes = [p]
    lib.gs_plan_pixels.restype = C.c_int64
    lib.gs_ce_update.argtypes = [C.c_int64, p, p, p]
    lib.gs_ce_update.restype = s
    lib.gs_prune_mask.argtypes = [p, p, C.c_int64, p, C.c_double, p, p]
    lib.gs_prune_mask.restype = s
    lib.gs_compact_points.argtypes = [p, p, C.c_int64, s, p, p, p, p, p]
    lib.gs_compact_points.restype = s
    lib.gs_weighted_scale.argtypes = [C.c_int64, p, p, C.c_float, C.c_float, p, p, p]
    lib.gs_weighted_scale.restype = s
    lib.gs_peak_probe.argtypes = [s, s, p, p, p]
    lib.gs_peak_probe.restype = s
    lib.gs_sort_pairs_static.argtypes = [p, p, C.c_int64, s, p, p, p]
    lib.gs_sort_pairs_static.restype = s
    lib.gs_sort_pairs_static_status.argtypes = [p, p]
    lib.gs_sort_pairs_static_status.restype = s
    lib.gs_sort_is_cooperative.argtypes = []
    lib.gs_sort_is_cooperative.restype = s
    lib.gs_hvsq_scratch_size.argtypes = [s, s]
    lib.gs_hvsq_scratch_size.restype = C.c_size_t
    lib.gs_hvsq.argtypes = [p, p, s, s, C.c_float, C.c_float, C.c_float, p, s, p, s, s, p,
                            C.c_size_t, p, p, p]
    lib.gs_hvsq.restype = s
    return lib


_lib = _load()


def lib():
    return _lib


def library_path() -> str:
    return _build.LIB


def _check(code, what):
    if code != GS_OK:
        raise GsError(code, what)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def cams_host(cams: np.ndarray):
    """(V, 20) float32 packed cameras -> ctypes array of gs_camera."""
    cams = np.asarray(cams, np.float32).reshape(-1, 20)
    arr = (gs_camera * len(cams))()
    for v, row in enumerate(cams):
        c = arr[v]
        for k in range(9):
            c.R[k] = float(row[k])
        for k in range(3):
            c.t[k] = float(row[9 + k])
        c.fx, c.fy, c.cx, c.cy = (float(x) for x in row[12:16])
        c.width, c.height = int(row[16]), int(row[17])
        c.znear, c.zfar = float(row[18]), float(row[19])
    return arr


def cams_device(cams: np.ndarray, device="cuda") -> torch.Tensor:
    """(V, 20) float32 packed cameras -> device bytes laid out as gs_camera[V]."""
    h = cams_host(cams)
    raw = np.frombuffer(bytes(h), np.uint8).copy()
    return torch.from_numpy(raw).to(device)


# --------------------------------------------------------------------------
# C-ABI wrappers with the library's names
# --------------------------------------------------------------------------
def gs_plan_init(plan_buf, n, sh_degree, cams_h, n_views, cfg):
    _check(_lib.gs_plan_init(plan_buf, n, sh_degree, cams_h, n_views, C.byref(cfg)),
           "gs_plan_init")


def gs_project(plan_buf, ws, scene, cams_d, fov, stream=None):
    _check(_lib.gs_project(plan_buf, _ptr(ws), ws.numel() * ws.element_size(), C.byref(scene),
                           _ptr(cams_d), C.byref(fov) if fov is not None else None,
                           _stream(stream)), "gs_project")


def gs_bin_sort(plan_buf, ws, stream=None):
    _check(_lib.gs_bin_sort(plan_buf, _ptr(ws), _stream(stream)), "gs_bin_sort")


def gs_render(plan_buf, ws, bg, rgb, T, last, stats=None, stream=None):
    bgv = (C.c_float * 3)(*[float(x) for x in bg])
    _check(_lib.gs_render(plan_buf, _ptr(ws), bgv, _ptr(rgb), _ptr(T), _ptr(last), _ptr(stats),
                          _stream(stream)), "gs_render")


def gs_render_fov(plan_buf, ws, bg, rgb, T, last, stats=None, stream=None):
    bgv = (C.c_float * 3)(*[float(x) for x in bg])
    _check(_lib.gs_render_fov(plan_buf, _ptr(ws), bgv, _ptr(rgb), _ptr(T), _ptr(last),
                              _ptr(stats), _stream(stream)), "gs_render_fov")


def gs_render_backward(plan_buf, ws, dL, T, last, bg, d_means, d_scales, d_quats, d_opac, d_sh,
                       d_opac_lv=None, d_dc_lv=None, stream=None):
    bgv = (C.c_float * 3)(*[float(x) for x in bg])
    _check(_lib.gs_render_backward(plan_buf, _ptr(ws), _ptr(dL), _ptr(T), _ptr(last), bgv,
                                   _ptr(d_means), _ptr(d_scales), _ptr(d_quats), _ptr(d_opac),
                                   _ptr(d_sh), _ptr(d_opac_lv), _ptr(d_dc_lv), _stream(stream)),
           "gs_render_backward")


def gs_ce_update(n, stats, ce_max, stream=None):
    _check(_lib.gs_ce_update(n, _ptr(stats), _ptr(ce_max), _stream(stream)), "gs_ce_update")


def gs_prune_mask(plan_buf, ws, n, ce_max, fraction, keep, stream=None):
    _check(_lib.gs_prune_mask(plan_buf, _ptr(ws), n, _ptr(ce_max), float(fraction), _ptr(keep),
                              _stream(stream)), "gs_prune_mask")


def gs_compact_points(plan_buf, ws, n, sh_degree, keep, scene_in, scene_out, n_out, stream=None):
    _check(_lib.gs_compact_points(plan_buf, _ptr(ws), n, sh_degree, _ptr(keep), C.byref(scene_in),
                                  C.byref(scene_out), _ptr(n_out), _stream(stream)),
           "gs_compact_points")


def gs_weighted_scale(n, scales, stats, T, gamma, ws_out, d_scales=None, stream=None):
    _check(_lib.gs_weighted_scale(n, _ptr(scales), _ptr(stats), float(T), float(gamma),
                                  _ptr(ws_out), _ptr(d_scales), _stream(stream)),
           "gs_weighted_scale")


def gs_peak_probe(kind, iters, sink, stream=None) -> int:
    """Launches the FMA (kind 0) or ex2 (kind 1) issue-rate probe; returns
    the lane operations launched (time the call with CUDA events)."""
    ops = C.c_int64(0)
    _check(_lib.gs_peak_probe(int(kind), int(iters), _ptr(sink), C.byref(ops), _stream(stream)),
           "gs_peak_probe")
    return int(ops.value)


class HvsqView:
    """Scratch and geometry of the HVSQ of one view (Sec. 2.2): width x
    height image, gaze pixel, focal length (pixels), quality rings (tangents,
    ``ring_tan``, the regions of Sec. 4.3) and the pooling law's tangent
    thresholds (``pool_tan``, ``r_base``: synth.pooling_tangents)."""

    def __init__(self, width, height, gaze, focal, ring_tan, pool_tan, r_base, device="cuda"):
        self.W, self.H = int(width), int(height)
        self.gaze = (float(gaze[0]), float(gaze[1]))
        self.focal = float(focal)
        self.ring_tan = np.ascontiguousarray(ring_tan, np.float32)
        self.pool_tan = np.ascontiguousarray(pool_tan, np.float32)
        self.r_base = int(r_base)
        nb = int(_lib.gs_hvsq_scratch_size(self.W, self.H))
        if nb == 0:
            raise GsError(GS_ERR_INVALID_ARG, "gs_hvsq_scratch_size")
        self.scratch = torch.empty(nb, dtype=torch.uint8, device=device)
        self.n_regions = len(self.ring_tan) + 1

    def __call__(self, alt, ref, out, d_alt=None, stream=None):
        """HVSQ per region into ``out`` (device float64, n_regions); the
        gradient of their sum into ``d_alt`` (device (W*H, 3)) if given."""
        rt = self.ring_tan.ctypes.data if len(self.ring_tan) else None
        pt = self.pool_tan.ctypes.data if len(self.pool_tan) else None
        _check(_lib.gs_hvsq(_ptr(alt), _ptr(ref), self.W, self.H, self.gaze[0], self.gaze[1],
                            self.focal, rt, len(self.ring_tan), pt, len(self.pool_tan),
                            self.r_base, _ptr(self.scratch), self.scratch.numel(), _ptr(out),
                            _ptr(d_alt), _stream(stream)), "gs_hvsq")


def gs_get_error(plan_buf, ws, stream=None):
    c = gs_counters()
    code = _lib.gs_get_error(plan_buf, _ptr(ws), _stream(stream), C.byref(c))
    return code, c


# --------------------------------------------------------------------------
# Renderer: plan + workspace + outputs
# --------------------------------------------------------------------------
class Renderer:
    """One plan (scene size, views, options) and its device workspace.

    ``scene_t``: dict of device tensors means/scales/quats/opac/sh;
    ``cams``: (V, 20) packed float32 cameras (numpy).
    Options map to ``gs_config``: ``tile`` 16 or 8; ``foveated`` reserves the
    foveation state; ``backward`` the gradient scratch; ``tight`` the
    opacity-aware tight support (same image, fewer pairs); ``multi_model`` a
    separate model per foveation level (implies ``foveated``); ``chunk`` /
    ``chunk_slots`` the heavy-tile chunked render; ``radix_bits`` the pair
    sort's digit width; ``max_pairs`` the pair capacity (``fit`` grows it);
    ``wait_spins`` the polls of the projection's bounded waits (0 = default,
    < 0 = give up at once, which exercises the timeout path).
    """

    def __init__(self, n, sh_degree, cams, tile=16, foveated=False, backward=False,
                 max_pairs=0, max_levels=0, chunk=0, radix_bits=0, chunk_slots=0,
                 tight=False, multi_model=False, wait_spins=0, device="cuda"):
        self.n, self.sh_degree = int(n), int(sh_degree)
        self.cams_np = np.asarray(cams, np.float32).reshape(-1, 20)
        self.V = len(self.cams_np)
        self.device = device
        self.cfg = gs_config(tile, chunk, (GS_FLAG_FOVEATED if foveated else 0)
                             | (GS_FLAG_BACKWARD if backward else 0)
                             | (GS_FLAG_TIGHT if tight else 0)
                             | (GS_FLAG_MULTI_MODEL | GS_FLAG_FOVEATED if multi_model else 0),
                             max_levels,
                             radix_bits, chunk_slots, max_pairs, wait_spins, 0)
        self.plan = C.create_string_buffer(int(_lib.gs_plan_size()))
        self._cams_h = cams_host(self.cams_np)
        gs_plan_init(self.plan, self.n, self.sh_degree, self._cams_h, self.V, self.cfg)
        self.ws_bytes = int(_lib.gs_workspace_size(self.plan))
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)
        self.cams_d = cams_device(self.cams_np, device)
        self.P = int(_lib.gs_plan_pixels(self.plan))
        self.T_tiles = int(_lib.gs_plan_tiles(self.plan))
        self.tile = tile
        self._keep = None

    # -- stages ------------------------------------------------------------
    def set_cameras(self, cams):
        cams = np.asarray(cams, np.float32).reshape(-1, 20)
        assert cams.shape == self.cams_np.shape
        self.cams_np = cams
        self.cams_d.copy_(cams_device(cams, self.device))

    def project(self, sc: dict, fov: dict | None = None, stream=None):
        scene = gs_scene(self.n, self.sh_degree, 0, sc["means"].data_ptr(),
                         sc["scales"].data_ptr(), sc["quats"].data_ptr(), sc["opac"].data_ptr(),
                         sc["sh"].data_ptr())
        f = None
        if fov is not None:
            f = gs_fov()
            f.n_levels = int(fov["n_levels"])
            f.band_px = float(fov["band_px"])
            for k, v in enumerate(np.asarray(fov["ring_tan"], np.float32)):
                f.ring_tan[k] = float(v)
            f.bound_m = fov["bound_m"].data_ptr()
            f.gaze_px = fov["gaze"].data_ptr()
            f.view_fov = fov["view_fov"].data_ptr() if fov.get("view_fov") is not None else None
            f.opacity_lv = fov["opacity_lv"].data_ptr() if fov.get("opacity_lv") is not None else None
            f.dc_lv = fov["dc_lv"].data_ptr() if fov.get("dc_lv") is not None else None
        self._keep = (sc, fov)   # the plan records these pointers
        gs_project(self.plan, self.ws, scene, self.cams_d, f, stream)

    def bin_sort(self, stream=None):
        gs_bin_sort(self.plan, self.ws, stream)

    # -- efficiency-aware pruning (Sec. 3.2-3.4) -----------------------------
    def _scene(self, sc: dict, n=None):
        return gs_scene(self.n if n is None else n, self.sh_degree, 0, sc["means"].data_ptr(),
                        sc["scales"].data_ptr(), sc["quats"].data_ptr(), sc["opac"].data_ptr(),
                        sc["sh"].data_ptr())

    def prune_mask(self, ce_max, fraction, stream=None):
        """uint8 keep mask: 0 for the floor(fraction * N) lowest-CE points.
        Overwrites the plan's depth order (project again before rendering)."""
        keep = torch.empty(self.n, dtype=torch.uint8, device=self.device)
        gs_prune_mask(self.plan, self.ws, self.n, ce_max, fraction, keep, stream)
        return keep

    def compact(self, sc: dict, keep, stream=None) -> dict:
        """The scene's kept points, in order (device tensors)."""
        out = {k: torch.empty_like(v) for k, v in sc.items()}
        n_out = torch.zeros(1, dtype=torch.int64, device=self.device)
        gs_compact_points(self.plan, self.ws, self.n, self.sh_degree, keep, self._scene(sc),
                          self._scene(out), n_out, stream)
        k = int(n_out.item())
        return {kk: v[:k] for kk, v in out.items()}

    def _replan(self, max_pairs):
        self.cfg.max_pairs = int(max_pairs)
        gs_plan_init(self.plan, self.n, self.sh_degree, self._cams_h, self.V, self.cfg)
        self.ws_bytes = int(_lib.gs_workspace_size(self.plan))
        self.ws = None
        torch.cuda.empty_cache()
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)

    def fit(self, sc: dict, fov: dict | None = None, headroom=1.15, stream=None):
        """project + bin_sort; if the pairs overflow the plan's capacity,
        re-plan with room for K * headroom pairs and run both again.  Returns
        the counters (synchronises)."""
        for _ in range(2):
            self.project(sc, fov, stream)
            self.bin_sort(stream)
            code, c = self.counters(stream)
            if code != GS_ERR_CAPACITY:
                break
            self._replan(int(c["n_pairs"] * headroom) + 1024)
        if code != GS_OK:
            raise GsError(code, "fit")
        return c

    def alloc_outputs(self, fov=False, stats=False):
        P = self.P
        k = 2 if fov else 1
        out = {"rgb": torch.empty(P, 3, device=self.device),
               "T": torch.empty(P * k, device=self.device),
               "last": torch.empty(P * k, dtype=torch.int32, device=self.device)}
        if stats:
            out["stats"] = torch.empty(4, self.n, dtype=torch.int32, device=self.device)
        return out

    def render(self, out, bg=(0, 0, 0), fov=False, stream=None):
        fn = gs_render_fov if fov else gs_render
        fn(self.plan, self.ws, bg, out["rgb"], out["T"], out["last"], out.get("stats"), stream)

    def backward(self, dL, out, grads, bg=(0, 0, 0), stream=None):
        gs_render_backward(self.plan, self.ws, dL, out["T"], out["last"], bg, grads["means"],
                           grads["scales"], grads["quats"], grads["opac"], grads["sh"],
                           grads.get("opac_lv"), grads.get("dc_lv"), stream)

    def launches_per_frame(self, fov=False, stats=False):
        """Kernels of this library launched by project + bin_sort + render."""
        tile_bits = max(1, int(self.T_tiles - 1).bit_length())
        want = self.cfg.radix_bits or 8
        passes = min(4, (tile_bits + want - 1) // want)
        # views, levels (+ level rows), project, pair count
        project = 1 + (2 if fov else 0) + (2 if self.n > 0 else 0)
        # depth sort (one cooperative launch, or hist, scan and 4 passes of
        # upsweep + scan + downsweep), offsets (upsweep, downsweep), emit +
        # large-item emit, pair sort (one cooperative launch that also marks
        # the tile ranges, or scan + 3 kernels per pass and a ranges kernel)
        if _lib.gs_sort_is_cooperative():
            sort = 0 if self.n == 0 else 1 + 2 + 2 + 1
        else:
            sort = 0 if self.n == 0 else (2 + 4 * 3) + 2 + 2 + (1 + 3 * passes) + 1
        render = 1 + (1 if stats and self.n > 0 else 0)
        if self.cfg.chunk > 0 and not stats and self.T_tiles > 0:
            render += 1     # work list of the chunked render
        return project + sort + render

    def counters(self, stream=None):
        code, c = gs_get_error(self.plan, self.ws, stream)
        return code, {"status": c.status, "n_visible": c.n_visible, "n_pairs": c.n_pairs,
                      "n_nonfinite": c.n_nonfinite, "n_evals": c.n_evals,
                      "n_blends": c.n_blends}

    def clear_error(self, stream=None):
        _check(_lib.gs_clear_error(self.plan, _ptr(self.ws), _stream(stream)), "gs_clear_error")

    # -- debug views of the workspace ----------------------------------------
    def region(self, rid, dtype, count):
        off, nb = C.c_size_t(), C.c_size_t()
        _check(_lib.gs_ws_region(self.plan, rid, C.byref(off), C.byref(nb)), "gs_ws_region")
        esz = torch.empty(0, dtype=dtype).element_size()
        return self.ws[off.value: off.value + count * esz].view(dtype)

    def sorted_pairs(self, K, stream=None):
        pt, pi = C.c_void_p(), C.c_void_p()
        _check(_lib.gs_sorted_pairs(self.plan, _ptr(self.ws), _stream(stream), C.byref(pt),
                                    C.byref(pi)), "gs_sorted_pairs")
        base = self.ws.data_ptr()
        ot, oi = pt.value - base, pi.value - base
        return (self.ws[ot: ot + 4 * K].view(torch.int32), self.ws[oi: oi + 4 * K].view(torch.int32))


def scene_to_device(scene, device="cuda") -> dict:
    """numpy Scene (synth.Scene) -> dict of contiguous device tensors."""
    return {"means": torch.from_numpy(np.ascontiguousarray(scene.means, np.float32)).to(device),
            "scales": torch.from_numpy(np.ascontiguousarray(scene.scales, np.float32)).to(device),
            "quats": torch.from_numpy(np.ascontiguousarray(scene.quats, np.float32)).to(device),
            "opac": torch.from_numpy(np.ascontiguousarray(scene.opac, np.float32)).to(device),
            "sh": torch.from_numpy(np.ascontiguousarray(scene.sh, np.float32)).to(device)}


def fov_to_device(f, device="cuda", opacity_lv=None, dc_lv=None) -> dict | None:
    if f is None:
        return None
    op = f.opacity_lv if opacity_lv is None else opacity_lv
    dc = f.dc_lv if dc_lv is None else dc_lv
    t = lambda a, dt: None if a is None else torch.from_numpy(np.ascontiguousarray(a, dt)).to(device)  # noqa: E731
    return {"n_levels": int(f.n_levels), "band_px": float(f.band_px),
            "ring_tan": np.asarray(f.ring_tan, np.float32), "bound_m": t(f.bound_m, np.uint8),
            "gaze": t(f.gaze, np.float32), "view_fov": t(f.view_fov, np.uint8),
            "opacity_lv": t(op, np.float32), "dc_lv": t(dc, np.float32)}
