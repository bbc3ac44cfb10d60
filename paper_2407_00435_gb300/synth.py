"""Seeded synthetic scenes, cameras and foveation inputs.

This module only draws random inputs; it holds none of the renderer's
arithmetic.  Both the CUDA path and the FP64 oracle consume exactly the arrays
it returns, so they see identical bytes.

Workload shapes follow the paper's statement of its rendering problem: each
point carries a position, per-axis scales, an orientation, an opacity and
spherical-harmonic colour coefficients (Sec. 2.1, "General PBNR Pipeline"),
"about 60" parameters per point for degree-3 SH (Sec. 7.4), per-tile
intersection counts spread over more than three orders of magnitude
(Sec. 5.2, Fig. 9), four nested quality levels (Sec. 4.2, Sec. 6).  The paper's
datasets and trained models are not available, so these generators stand in
for them.

All arrays are C-contiguous ``float32`` (or ``uint8``) numpy arrays:

* ``means``  (N, 3)      world positions
* ``scales`` (N, 3)      per-axis standard deviations (already activated, > 0)
* ``quats``  (N, 4)      rotation quaternions (w, x, y, z), unit length
* ``opac``   (N,)        opacities in (0, 1) (already activated)
* ``sh``     (N, S, 3)   SH coefficients, S = (degree + 1)^2, RGB last
* cameras    (V, 20)     see :func:`camera_lookat` for the packing
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Normalisation of the degree-0 real spherical harmonic, 1 / (2 sqrt(pi)).
# Used only to turn a desired RGB colour into a DC coefficient.
_Y00 = 0.5 / math.sqrt(math.pi)

CAM_FIELDS = 20  # R[9], t[3], fx, fy, cx, cy, width, height, znear, zfar


@dataclass
class Scene:
    means: np.ndarray
    scales: np.ndarray
    quats: np.ndarray
    opac: np.ndarray
    sh: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])


@dataclass
class Foveation:
    """Inputs of the foveated multi-level render (Sec. 4.1-4.2)."""
    n_levels: int
    bound_m: np.ndarray           # (N,) uint8 in 1..L, highest level using the point
    ring_tan: np.ndarray          # (L-1,) float32, tan of ring eccentricities, ascending
    band_px: float                # width of the blend band outside each ring, pixels
    gaze: np.ndarray              # (V, 2) float32 gaze pixel per view
    view_fov: np.ndarray | None = None   # (V,) uint8, 1 = foveated view, 0 = plain
    opacity_lv: np.ndarray | None = None  # (L-1, N) float32, levels 2..L
    dc_lv: np.ndarray | None = None       # (L-1, N, 3) float32, levels 2..L
    disjoint: bool = False        # bound_m is each point's model level (one model per level)


@dataclass
class Workload:
    name: str
    scene: Scene
    cams: np.ndarray              # (V, 20) float32
    tile: int = 16
    fov: Foveation | None = None
    meta: dict = field(default_factory=dict)


# --------------------------------------------------------------------------
# cameras
# --------------------------------------------------------------------------
def camera_lookat(eye, target, width, height, fov_y_deg=60.0, znear=0.2,
                  zfar=1000.0, down=(0.0, 1.0, 0.0)) -> np.ndarray:
    """Pinhole camera as a packed float32 row.

    Convention (OpenCV): camera x right, y down, z forward.  ``R`` maps world
    to camera (rows are the camera axes in world coordinates), ``t = -R eye``.
    Vertical field of view ``fov_y_deg``, square pixels, principal point at
    the image centre.  Packing: R (row-major, 9), t (3), fx, fy, cx, cy,
    width, height, znear, zfar.
    """
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    fwd = target - eye
    fwd /= np.linalg.norm(fwd)
    d = np.asarray(down, np.float64)
    d = d - d.dot(fwd) * fwd
    if np.linalg.norm(d) < 1e-9:  # looking straight along `down`
        d = np.array([0.0, 0.0, 1.0]) - fwd[2] * fwd
    d /= np.linalg.norm(d)
    right = np.cross(d, fwd)
    R = np.stack([right, d, fwd])
    t = -R @ eye
    fy = 0.5 * height / math.tan(math.radians(fov_y_deg) * 0.5)
    row = np.concatenate([R.reshape(-1), t,
                          [fy, fy, 0.5 * width, 0.5 * height, width, height,
                           znear, zfar]])
    return row.astype(np.float32)


def orbit_cameras(rng, n_views, radius, sizes, fov_y_deg=60.0):
    """Views on a sphere of ``radius`` looking at the origin.

    ``sizes`` is a list of (width, height) per view.
    """
    cams = []
    for v in range(n_views):
        while True:
            p = rng.standard_normal(3)
            if np.linalg.norm(p) > 1e-3:
                break
        p = p / np.linalg.norm(p) * radius
        w, h = sizes[v]
        cams.append(camera_lookat(p, (0, 0, 0), w, h, fov_y_deg))
    return np.stack(cams)


# --------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------
def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4)).astype(np.float64)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _sh_coeffs(rng, n, degree, dc_mode):
    S = (degree + 1) ** 2
    sh = np.empty((n, S, 3), np.float32)
    if dc_mode == "rgb":
        # DC chosen so that the degree-0 colour is uniform in [0, 1].
        rgb = rng.uniform(0.0, 1.0, (n, 3))
        sh[:, 0, :] = (rgb - 0.5) / _Y00
    else:
        sh[:, 0, :] = rng.uniform(0.0, 1.0, (n, 3))
    if S > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.05, (n, S - 1, 3))
    return sh


def uniform_scene(rng, n, degree=0, log_scale=(-3.5, 0.5), opac_std=1.0,
                  dc_mode="rgb") -> Scene:
    """Means uniform in [-1, 1]^3, log-normal scales, random unit quaternions,
    opacity = sigmoid(N(0, opac_std))."""
    means = rng.uniform(-1.0, 1.0, (n, 3)).astype(np.float32)
    scales = np.exp(rng.normal(log_scale[0], log_scale[1], (n, 3))).astype(np.float32)
    quats = _unit_quats(rng, n)
    opac = _sigmoid(rng.normal(0.0, opac_std, n)).astype(np.float32)
    sh = _sh_coeffs(rng, n, degree, dc_mode)
    return Scene(means, scales, quats, opac, sh, degree)


def _random_rotations(rng, k):
    """Haar-random rotation matrices from the QR factorisation of Gaussian
    matrices (signs fixed so that det = +1)."""
    a = rng.standard_normal((k, 3, 3))
    q, r = np.linalg.qr(a)
    d = np.sign(np.diagonal(r, axis1=1, axis2=2))
    d[d == 0] = 1.0
    q = q * d[:, None, :]
    neg = np.linalg.det(q) < 0
    q[neg, :, 0] *= -1.0
    return q


# Blob mixture calibration: blob axis standard deviations are log-uniform in
# [BLOB_STD_LO, BLOB_STD_HI] and blob k gets weight (k + 1)^-BLOB_ZIPF.  The
# values were chosen so that the 1920x1080, 1M-point workload has a heavy
# tailed per-tile count: 16x16-tile counts p10 ~220, median ~720, max ~5.1k,
# K ~ 9.4M tile/point pairs.
BLOB_STD_LO = 0.5
BLOB_STD_HI = 2.0
BLOB_ZIPF = 0.3


def blob_scene(rng, n, n_blobs=200, degree=3, log_scale=(-4.5, 0.7),
               opac_std=1.5, chunk=1 << 20) -> Scene:
    """Mixture of anisotropic Gaussian blobs (heavy-tailed depth complexity).

    Centres uniform in [-1, 1]^3, random rotation per blob, per-axis blob
    std log-uniform, Zipf-like blob weights.  Point scales log-normal,
    opacity sigmoid(N(0, opac_std)), SH DC ~ U[0, 1], higher orders
    ~ N(0, 0.05).
    """
    centres = rng.uniform(-1.0, 1.0, (n_blobs, 3))
    rots = _random_rotations(rng, n_blobs)
    stds = np.exp(rng.uniform(math.log(BLOB_STD_LO), math.log(BLOB_STD_HI),
                              (n_blobs, 3)))
    w = (np.arange(n_blobs) + 1.0) ** -BLOB_ZIPF
    w = rng.permutation(w)
    w /= w.sum()
    which = rng.choice(n_blobs, size=n, p=w)
    means = np.empty((n, 3), np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        k = which[s:e]
        z = rng.standard_normal((e - s, 3)) * stds[k]
        means[s:e] = (centres[k] + np.einsum("nij,nj->ni", rots[k], z)).astype(np.float32)
    scales = np.exp(rng.normal(log_scale[0], log_scale[1], (n, 3))).astype(np.float32)
    quats = _unit_quats(rng, n)
    opac = _sigmoid(rng.normal(0.0, opac_std, n)).astype(np.float32)
    sh = _sh_coeffs(rng, n, degree, "coef")
    return Scene(means, scales, quats, opac, sh, degree)


def nested_levels(rng, n, n_levels=4):
    """Quality bound m per point from a seeded rank (strict subsetting,
    Sec. 4.2): level k holds the first N / 2^(k-1) points of a random
    permutation, so m = 4 for rank < N/8, 3 for < N/4, 2 for < N/2, else 1."""
    rank = np.empty(n, np.int64)
    rank[rng.permutation(n)] = np.arange(n)
    m = np.ones(n, np.uint8)
    for k in range(2, n_levels + 1):
        m[rank < n / (2 ** (k - 1))] = k
    return m


def ring_tangents(ring_deg):
    return np.tan(np.radians(np.asarray(ring_deg, np.float64))).astype(np.float32)


def pooling_tangents(r0=1.0, k=0.025, r_max=64):
    """Tangents of the eccentricities (degrees) at which a pooling half-width
    r0 + k e^2 reaches floor(r0) + 1, ..., r_max: the thresholds of the HVSQ
    pooling law (Sec. 2.2), float32, ascending.  Returns (tangents, r_base)."""
    base = int(math.floor(r0))
    out = []
    for j in range(base + 1, int(r_max) + 1):
        e = math.sqrt((j - r0) / k)
        if e >= 89.0:
            break
        out.append(math.tan(math.radians(e)))
    return np.asarray(out, np.float32), base


def random_gaze(rng, cams):
    """Gaze pixel per view, uniform in the central 50% of each axis."""
    w = cams[:, 16].astype(np.float64)
    h = cams[:, 17].astype(np.float64)
    gx = rng.uniform(0.25, 0.75, len(cams)) * w
    gy = rng.uniform(0.25, 0.75, len(cams)) * h
    return np.stack([gx, gy], 1).astype(np.float32)


def multiversion_params(rng, scene: Scene, n_levels):
    """Per-level opacity and SH DC for levels 2..L (selective
    multi-versioning, Sec. 4.2): small perturbations of the shared values."""
    n = scene.n
    op = np.clip(scene.opac[None, :] * rng.uniform(0.7, 1.0, (n_levels - 1, n)),
                 1e-3, 0.999).astype(np.float32)
    dc = (scene.sh[None, :, 0, :] + rng.normal(0, 0.1, (n_levels - 1, n, 3))).astype(np.float32)
    return op, dc


def multi_model_scene(rng, scene: Scene, bound_m, n_levels):
    """Separate per-level models for the multi-model foveated render
    (Sec. 4.1, main pipeline; the paper's multi-model baseline prunes each
    level's model from the level-1 model on its own).  Level 1 is `scene`;
    level l >= 2 is a copy of the points of the nested level-l subset
    (bound_m >= l) with parameters of its own: opacity and SH DC perturbed as
    in multiversion_params, scales by a log-normal factor.  Returns the
    concatenated scene and the uint8 model level of every point."""
    parts = [(np.arange(scene.n), 1)]
    for lvl in range(2, n_levels + 1):
        parts.append((np.nonzero(np.asarray(bound_m) >= lvl)[0], lvl))
    means, scales, quats, opac, sh, level = [], [], [], [], [], []
    for idx, lvl in parts:
        k = len(idx)
        means.append(scene.means[idx])
        quats.append(scene.quats[idx])
        if lvl == 1:
            scales.append(scene.scales[idx])
            opac.append(scene.opac[idx])
            sh.append(scene.sh[idx])
        else:
            scales.append((scene.scales[idx] * np.exp(rng.normal(0.0, 0.1, (k, 1)))).astype(np.float32))
            opac.append(np.clip(scene.opac[idx] * rng.uniform(0.7, 1.0, k), 1e-3, 0.999).astype(np.float32))
            shl = scene.sh[idx].copy()
            shl[:, 0, :] += rng.normal(0, 0.1, (k, 3)).astype(np.float32)
            sh.append(shl)
        level.append(np.full(k, lvl, np.uint8))
    sc = Scene(np.concatenate(means), np.concatenate(scales), np.concatenate(quats),
               np.concatenate(opac), np.concatenate(sh), scene.sh_degree)
    return sc, np.concatenate(level)


def multi_model_workload(n=None, views=None) -> Workload:
    """The foveated stereo workload with a separate model per level: the
    level-l model is its own copy of the nested level-l subset (N, N/2, N/4,
    N/8 points, 1.875 N in all), same rings, band and gaze."""
    wl = workload(2, n=n, views=views)
    rng = np.random.default_rng(config_seed(2) + 100)
    sc, lv = multi_model_scene(rng, wl.scene, wl.fov.bound_m, wl.fov.n_levels)
    f = wl.fov
    fov = Foveation(f.n_levels, lv, f.ring_tan, f.band_px, f.gaze, f.view_fov, disjoint=True)
    name = wl.name.replace("fov_stereo", "mmfr_stereo")
    return Workload(name, sc, wl.cams, wl.tile, fov)


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------
def fov_fwd_bwd_workload(n=None, views=None) -> Workload:
    """The forward + backward workload (500k points, SH3, 8 views of 1024^2
    on the orbit, L1 loss) with each view foveated as in the stereo workload:
    4 nested levels by a seeded rank (100/50/25/12.5 % of the points), rings
    at 10/20/35 degrees, a 32-px blend band, a gaze per view uniform in the
    central 50 %.  Retraining through the foveated renderer (Sec. 4.3)."""
    wl = workload(3, n=n, views=views)
    rng = np.random.default_rng(config_seed(3) + 200)
    m = nested_levels(rng, wl.scene.n, 4)
    gaze = random_gaze(rng, wl.cams)
    fov = Foveation(4, m, ring_tangents([10, 20, 35]), 32.0, gaze)
    return Workload(wl.name.replace("fwd_bwd", "fov_fwd_bwd"), wl.scene, wl.cams, wl.tile, fov)


def config_seed(idx: int) -> int:
    return 1000 + idx


def workload(idx: int, n=None, views=None) -> Workload:
    """Workload ``idx`` (0..4).  ``n``/``views`` shrink a workload for tests."""
    rng = np.random.default_rng(config_seed(idx))
    if idx == 0:
        # plain forward, 1 view: 10k points, SH0, 128x128, 60 deg FOV
        N = n or 10_000
        sc = uniform_scene(rng, N, degree=0, log_scale=(-3.5, 0.5), opac_std=1.0,
                           dc_mode="rgb")
        cams = camera_lookat((0, 0, -4), (0, 0, 0), 128, 128)[None]
        return Workload("plain_128x128_n10k_sh0", sc, cams, 16)
    if idx == 1:
        # plain forward at 1920x1080, 1M points, SH3, blob mixture
        N = n or 1_000_000
        sc = blob_scene(rng, N, 200, 3)
        cams = camera_lookat((0, 0, -4), (0, 0, 0), 1920, 1080)[None]
        return Workload("plain_1920x1080_n1M_sh3", sc, cams, 16)
    if idx == 2:
        # foveated stereo, 3M points, 2 eyes at 1920x1920, 4 nested levels
        N = n or 3_000_000
        sc = blob_scene(rng, N, 200, 3)
        side = views or 1920
        cams = np.stack([camera_lookat((dx, 0, -4), (dx, 0, 0), side, side)
                         for dx in (-0.032, 0.032)])
        m = nested_levels(rng, N, 4)
        g = random_gaze(rng, cams[:1])
        gaze = np.repeat(g, 2, axis=0)
        fov = Foveation(4, m, ring_tangents([10, 20, 35]), 32.0, gaze)
        return Workload("fov_stereo_2x1920x1920_n3M", sc, cams, 16, fov)
    if idx == 3:
        # forward + backward, 500k points, SH3, 8 views 1024^2 on an orbit
        N = n or 500_000
        sc = blob_scene(rng, N, 200, 3)
        V = views or 8
        cams = orbit_cameras(rng, V, 4.0, [(1024, 1024)] * V)
        return Workload("fwd_bwd_8x1024x1024_n500k", sc, cams, 16)
    if idx == 4:
        # 64 uneven views, mixed foveated/plain, 6M points, 600 blobs
        N = n or 6_000_000
        sc = blob_scene(rng, N, 600, 3)
        V = views or 64
        sides = rng.choice([256, 512, 1024, 1536, 2048], V)
        cams = orbit_cameras(rng, V, 4.0, [(int(s), int(s)) for s in sides])
        m = nested_levels(rng, N, 4)
        gaze = random_gaze(rng, cams)
        vf = (rng.uniform(size=V) < 0.5).astype(np.uint8)
        fov = Foveation(4, m, ring_tangents([10, 20, 35]), 32.0, gaze, vf)
        return Workload("batched_64views_uneven_n6M", sc, cams, 16, fov)
    raise ValueError(idx)
