"""FP64 CPU oracle for the tile rasterizer (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does.

The C source (``gs_oracle.c``) is compiled with gcc, without floating-point
contraction, into ``liboracle.so`` next to it; this module loads it with
ctypes and offers numpy-level wrappers.  Every function states the paper
passage it follows in ``gs_oracle.h``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# The same source built with -fopenmp: its independent per-item and per-pixel
# loops run on all host cores (same arithmetic per item and pixel).
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")

ORC_NVAL = 15
ORC_SUPP = 6            # tight-support record: keyed u, v, covariance a b c, tau
(ORC_U, ORC_V, ORC_CA, ORC_CB, ORC_CC, ORC_R, ORC_G, ORC_B, ORC_RR, ORC_RG,
 ORC_RB, ORC_DEPTH, ORC_SA, ORC_SB, ORC_SC) = range(15)


def _compile(out, extra):
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-Wall", "-Wno-unused-function", "-Wno-unknown-pragmas",
           *extra, _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)


def _stale(path):
    return (not os.path.exists(path)
            or os.path.getmtime(path) < max(os.path.getmtime(_SRC),
                                            os.path.getmtime(os.path.join(_HERE, "gs_oracle.h"))))


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, no FP contraction, no fast-math), the
    single-threaded library and its all-core (-fopenmp) build."""
    if force or _stale(_LIB):
        _compile(_LIB, [])
    if force or _stale(_LIB_OMP):
        try:
            _compile(_LIB_OMP, ["-fopenmp"])
        except subprocess.CalledProcessError:
            pass   # no OpenMP runtime: only the single-threaded build
    return _LIB


class _Cam(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float),
                ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32),
                ("znear", C.c_float), ("zfar", C.c_float)]


class _Fov(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("bound_m", C.c_void_p),
                ("ring_tan", C.c_void_p), ("band_px", C.c_float),
                ("gaze", C.c_void_p), ("view_fov", C.c_void_p),
                ("opacity_lv", C.c_void_p), ("dc_lv", C.c_void_p), ("disjoint", C.c_int32)]


_lib = None
_threads = False


def use_all_cores(on: bool = True) -> bool:
    """Switch the wrappers to the all-core build (True) or back to the
    single-threaded one.  Returns whether the all-core build is in use."""
    global _lib, _threads
    build()
    on = bool(on) and os.path.exists(_LIB_OMP)
    if on != _threads:
        _threads = on
        _lib = None
    return _threads


def threads() -> int:
    """Host threads the current build uses."""
    if not _threads:
        return 1
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_OMP if _threads else _LIB)
        p = C.c_void_p
        L.orc_keyed_project.argtypes = [C.c_int, p, p, p, p, p, C.c_int, C.c_int, p, C.c_int, p, p,
                                        p, p, p]
        L.orc_tile_levels.argtypes = [C.c_int, p, C.c_int, p, p]
        L.orc_total_tiles.argtypes = [C.c_int, p, C.c_int]
        L.orc_total_tiles.restype = C.c_int64
        L.orc_count_pairs.argtypes = [C.c_int, C.c_int, p, C.c_int, p, p, p, p, p, p]
        L.orc_count_pairs.restype = C.c_int64
        L.orc_bin.argtypes = [C.c_int, C.c_int, p, C.c_int, p, p, p, p, p, p, C.c_int64, p, p,
                              p]
        L.orc_project_values.argtypes = [C.c_int, p, p, p, p, C.c_int, C.c_int, p, p, p]
        L.orc_sh_basis.argtypes = [p, p]
        L.orc_sh_basis.restype = None
        L.orc_render.argtypes = [C.c_int, C.c_int, p, C.c_int, p, p, p, p, p, p, p,
                                 C.c_int64, p, p, p, p, p, p, p, p]
        L.orc_render_brute.argtypes = [C.c_int, C.c_int, p, C.c_int, p, p, p, p, p, p, p,
                                       p, p, p]
        L.orc_backward.argtypes = [C.c_int, p, p, p, p, p, C.c_int, C.c_int, p, C.c_int,
                                   p, p, p, p, p, p, p, p, p, p, p, p, p]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def cams_struct(cams: np.ndarray):
    cams = np.asarray(cams, np.float32).reshape(-1, 20)
    arr = (_Cam * len(cams))()
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


def view_dims(cams, tile):
    cams = np.asarray(cams).reshape(-1, 20)
    W = cams[:, 16].astype(np.int64)
    H = cams[:, 17].astype(np.int64)
    tx = (W + tile - 1) // tile
    ty = (H + tile - 1) // tile
    return W, H, tx, ty


@dataclass
class FovArrays:
    """numpy side of an orc_fov; keeps the arrays alive."""
    n_levels: int
    bound_m: np.ndarray
    ring_tan: np.ndarray
    band_px: float
    gaze: np.ndarray
    view_fov: np.ndarray | None = None
    opacity_lv: np.ndarray | None = None
    dc_lv: np.ndarray | None = None
    disjoint: bool = False   # a separate model per level (bound_m = model level)

    @staticmethod
    def from_synth(f, opacity_lv=None, dc_lv=None):
        if f is None:
            return None
        op = f.opacity_lv if opacity_lv is None else opacity_lv
        dc = f.dc_lv if dc_lv is None else dc_lv
        return FovArrays(
            int(f.n_levels), np.ascontiguousarray(f.bound_m, np.uint8),
            np.ascontiguousarray(f.ring_tan, np.float32), float(f.band_px),
            np.ascontiguousarray(f.gaze, np.float32),
            None if f.view_fov is None else np.ascontiguousarray(f.view_fov, np.uint8),
            None if op is None else np.ascontiguousarray(op, np.float64),
            None if dc is None else np.ascontiguousarray(dc, np.float64),
            bool(getattr(f, "disjoint", False)))

    def struct(self):
        s = _Fov()
        s.n_levels = self.n_levels
        s.bound_m = _ptr(self.bound_m)
        s.ring_tan = _ptr(self.ring_tan)
        s.band_px = self.band_px
        s.gaze = _ptr(self.gaze)
        s.view_fov = _ptr(self.view_fov)
        s.opacity_lv = _ptr(self.opacity_lv)
        s.dc_lv = _ptr(self.dc_lv)
        s.disjoint = 1 if self.disjoint else 0
        return s


def _c32(a):
    return np.ascontiguousarray(a, np.float32)


def _c64(a):
    return np.ascontiguousarray(a, np.float64)


def keyed_project(scene, cams, tile, tight=False, fov: "FovArrays | None" = None):
    """Keyed FP32 projection.  Returns (vis, depth bits, rect) and, with
    ``tight``, also the (V*N, 6) tight-support records."""
    n, V = scene.n, len(cams)
    vis = np.zeros(V * n, np.uint8)
    dbits = np.zeros(V * n, np.uint32)
    rect = np.zeros((V * n, 4), np.int32)
    supp = np.zeros((V * n, ORC_SUPP), np.float32) if tight else None
    cs = cams_struct(cams)
    fs = fov.struct() if fov is not None else None
    arrs = [_c32(scene.means), _c32(scene.scales), _c32(scene.quats), _c32(scene.opac),
            _c32(scene.sh)]
    lib().orc_keyed_project(n, *[a.ctypes.data for a in arrs], scene.sh_degree, V,
                            C.addressof(cs), tile, C.addressof(fs) if fs is not None else None,
                            vis.ctypes.data, dbits.ctypes.data, rect.ctypes.data, _ptr(supp))
    if tight:
        return vis, dbits, rect, supp
    return vis, dbits, rect


def tile_levels(cams, tile, fov: FovArrays | None):
    cs = cams_struct(cams)
    T = lib().orc_total_tiles(len(cams), C.addressof(cs), tile)
    out = np.zeros(T, np.uint8)
    fs = fov.struct() if fov is not None else None
    lib().orc_tile_levels(len(cams), C.addressof(cs), tile,
                          C.addressof(fs) if fs is not None else None, out.ctypes.data)
    return out


@dataclass
class Bins:
    vis: np.ndarray
    dbits: np.ndarray
    rect: np.ndarray
    tile_level: np.ndarray | None
    counts: np.ndarray
    keys: np.ndarray
    vals: np.ndarray
    ranges: np.ndarray  # (T, 2)
    supp: np.ndarray | None = None   # (V*N, 6) tight-support records, if used

    @property
    def K(self):
        return int(len(self.keys))


def bin_pairs(scene, cams, tile, fov: FovArrays | None = None, tight=False) -> Bins:
    """Keyed projection, FR filter, optional tight support, pair emission,
    stable sort, ranges."""
    kp = keyed_project(scene, cams, tile, tight=tight, fov=fov)
    vis, dbits, rect = kp[:3]
    supp = kp[3] if tight else None
    n, V = scene.n, len(cams)
    cs = cams_struct(cams)
    tl = tile_levels(cams, tile, fov) if fov is not None else None
    bm = fov.bound_m if fov is not None else None
    counts = np.zeros(V * n, np.uint32)
    K = lib().orc_count_pairs(n, V, C.addressof(cs), tile, vis.ctypes.data, rect.ctypes.data,
                              _ptr(tl), _ptr(bm), _ptr(supp), counts.ctypes.data)
    T = lib().orc_total_tiles(V, C.addressof(cs), tile)
    keys = np.zeros(K, np.uint64)
    vals = np.zeros(K, np.uint32)
    ranges = np.zeros((T, 2), np.uint32)
    rc = lib().orc_bin(n, V, C.addressof(cs), tile, vis.ctypes.data, dbits.ctypes.data,
                       rect.ctypes.data, _ptr(tl), _ptr(bm), _ptr(supp), K, keys.ctypes.data,
                       vals.ctypes.data, ranges.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"orc_bin failed: {rc}")
    return Bins(vis, dbits, rect, tl, counts, keys, vals, ranges, supp)


def project_values(scene, cams, vis, means=None, scales=None, quats=None, sh=None):
    n, V = scene.n, len(cams)
    out = np.zeros((V * n, ORC_NVAL), np.float64)
    cs = cams_struct(cams)
    m = _c64(scene.means if means is None else means)
    s = _c64(scene.scales if scales is None else scales)
    q = _c64(scene.quats if quats is None else quats)
    h = _c64(scene.sh if sh is None else sh)
    lib().orc_project_values(n, m.ctypes.data, s.ctypes.data, q.ctypes.data, h.ctypes.data,
                             scene.sh_degree, V, C.addressof(cs), vis.ctypes.data,
                             out.ctypes.data)
    return out


def sh_basis(d):
    d = _c64(d)
    Y = np.zeros(16, np.float64)
    lib().orc_sh_basis(d.ctypes.data, Y.ctypes.data)
    return Y


@dataclass
class Image:
    rgb: np.ndarray      # (P, 3)
    T: np.ndarray        # (P, 2)
    last: np.ndarray     # (P, 2)
    margin: np.ndarray   # (P,) smallest relative margin of any decision
    wband: np.ndarray    # (P,)
    ambB: np.ndarray     # (P,) what flipping the ambiguous decisions can change
    amb: np.ndarray      # (P,) bool: a decision inside its FP32 uncertainty window
    stats: np.ndarray | None  # (4, N)


def render(scene, cams, tile, bins: Bins, fov: FovArrays | None = None, bg=(0, 0, 0),
           pix=None, stats=False, vp=None, opac=None) -> Image:
    """Composite pixels (Eq. 1a); ``pix`` = global pixel ids or None (all)."""
    n, V = scene.n, len(cams)
    cs = cams_struct(cams)
    if vp is None:
        vp = project_values(scene, cams, bins.vis)
    op = _c64(scene.opac if opac is None else opac)
    W, H, _, _ = view_dims(cams, tile)
    P = int((W * H).sum()) if pix is None else len(pix)
    pix_arr = None if pix is None else np.ascontiguousarray(pix, np.int64)
    rgb = np.zeros((P, 3))
    T = np.zeros((P, 2))
    last = np.zeros((P, 2), np.int32)
    margin = np.zeros(P)
    wband = np.zeros(P)
    ambB = np.zeros(P)
    amb = np.zeros(P, np.uint8)
    st = np.zeros((4, n), np.uint32) if (stats and pix is None) else None
    fs = fov.struct() if fov is not None else None
    bgv = _c64(bg)
    rc = lib().orc_render(n, V, C.addressof(cs), tile, vp.ctypes.data, op.ctypes.data,
                          bins.vals.ctypes.data, bins.ranges.ctypes.data,
                          C.addressof(fs) if fs is not None else None, bgv.ctypes.data,
                          _ptr(pix_arr), P, rgb.ctypes.data, T.ctypes.data, last.ctypes.data,
                          margin.ctypes.data, wband.ctypes.data, ambB.ctypes.data,
                          amb.ctypes.data, _ptr(st))
    if rc != 0:
        raise RuntimeError(f"orc_render failed: {rc}")
    return Image(rgb, T, last, margin, wband, ambB, amb.astype(bool), st)


def render_brute(scene, cams, tile, fov: FovArrays | None = None, bg=(0, 0, 0)):
    """Per-pixel definition of Eq. 1 (no tile lists, no foveation tile
    filter).  Returns (rgb, T, last_item): last_item is the item v*N + i of
    the last blended point of each accumulator, -1 if none."""
    n, V = scene.n, len(cams)
    vis, dbits, rect = keyed_project(scene, cams, tile)
    vp = project_values(scene, cams, vis)
    cs = cams_struct(cams)
    W, H, _, _ = view_dims(cams, tile)
    P = int((W * H).sum())
    rgb = np.zeros((P, 3))
    T = np.zeros((P, 2))
    last = np.zeros((P, 2), np.int32)
    fs = fov.struct() if fov is not None else None
    op = _c64(scene.opac)
    bgv = _c64(bg)
    rc = lib().orc_render_brute(n, V, C.addressof(cs), tile, vis.ctypes.data, dbits.ctypes.data,
                                rect.ctypes.data, vp.ctypes.data, op.ctypes.data,
                                C.addressof(fs) if fs is not None else None, bgv.ctypes.data,
                                rgb.ctypes.data, T.ctypes.data, last.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"orc_render_brute failed: {rc}")
    return rgb, T, last


@dataclass
class Grads:
    means: np.ndarray
    scales: np.ndarray
    quats: np.ndarray
    opac: np.ndarray
    sh: np.ndarray
    opac_lv: np.ndarray | None
    dc_lv: np.ndarray | None
    # sum of |term| behind each element (same keys), or None
    mag: dict | None = None


class _GradMag(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("means", "scales", "quats", "opac", "sh", "opac_lv",
                                          "dc_lv")]


def backward(scene, cams, tile, bins: Bins, dL_drgb, fov: FovArrays | None = None,
             bg=(0, 0, 0), means=None, scales=None, quats=None, opac=None, sh=None) -> Grads:
    """Analytic FP64 gradient of sum(dL_drgb * rgb), binning held fixed."""
    n, V = scene.n, len(cams)
    S = (scene.sh_degree + 1) ** 2
    cs = cams_struct(cams)
    m = _c64(scene.means if means is None else means)
    s = _c64(scene.scales if scales is None else scales)
    q = _c64(scene.quats if quats is None else quats)
    o = _c64(scene.opac if opac is None else opac)
    h = _c64(scene.sh if sh is None else sh)
    g = _c64(dL_drgb)
    dm = np.zeros((n, 3)); ds = np.zeros((n, 3)); dq = np.zeros((n, 4)); do = np.zeros(n)
    dh = np.zeros((n, S, 3))
    L = fov.n_levels if fov is not None else 1
    dol = np.zeros((L - 1, n)) if (fov is not None and fov.opacity_lv is not None) else None
    ddl = np.zeros((L - 1, n, 3)) if (fov is not None and fov.dc_lv is not None) else None
    fs = fov.struct() if fov is not None else None
    bgv = _c64(bg)
    mag = {k: np.zeros_like(v) for k, v in (("means", dm), ("scales", ds), ("quats", dq),
                                            ("opac", do), ("sh", dh))}
    if dol is not None:
        mag["opac_lv"] = np.zeros_like(dol)
    if ddl is not None:
        mag["dc_lv"] = np.zeros_like(ddl)
    ms = _GradMag(*[_ptr(mag.get(k)) for k in ("means", "scales", "quats", "opac", "sh",
                                                "opac_lv", "dc_lv")])
    rc = lib().orc_backward(n, m.ctypes.data, s.ctypes.data, q.ctypes.data, o.ctypes.data,
                            h.ctypes.data, scene.sh_degree, V, C.addressof(cs), tile,
                            bins.vals.ctypes.data, bins.ranges.ctypes.data,
                            C.addressof(fs) if fs is not None else None, bgv.ctypes.data,
                            g.ctypes.data, dm.ctypes.data, ds.ctypes.data, dq.ctypes.data,
                            do.ctypes.data, dh.ctypes.data, _ptr(dol), _ptr(ddl),
                            C.addressof(ms))
    if rc != 0:
        raise RuntimeError(f"orc_backward failed: {rc}")
    return Grads(dm, ds, dq, do, dh, dol, ddl, mag)
