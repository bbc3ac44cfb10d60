"""Shared helpers of the GPU tests: run the CUDA path and the oracle on the
same seeded inputs and compare."""
import numpy as np

# Image tolerance of the forward path (per RGB channel, colours in [0, 1]).
IMG_MAX_ABS = 1e-3
IMG_MEAN_ABS = 1e-5
# A pixel whose alpha-floor or early-stop decision lies inside the
# uncertainty window of an FP32 evaluation (flagged by the oracle: alpha
# within 1e-4 relative of 1/255, against a derived FP32 alpha error below
# 4e-5; T (1 - alpha) within 1e-4 plus the running worst-case bound of T's
# FP32 relative error of 1e-4) may take the other branch; it is compared
# against what a flipped decision can change (the oracle's ambB:
# 2 T c_max / 255 per flipped floor decision, T c_max for the stop).
# Ambiguous pixels must stay a small minority of the compared pixels.
AMBIG_MAX_FRACTION = 0.02


def run_gpu(gs, wl, fov=None, stats=False, tile=None, bg=(0, 0, 0), mv=None, max_pairs=0,
            backward=False, chunk=0, chunk_slots=0, tight=False, multi_model=False):
    import torch
    sc = gs.scene_to_device(wl.scene)
    f = None
    if fov is not None:
        f = gs.fov_to_device(fov, opacity_lv=None if mv is None else mv[0],
                             dc_lv=None if mv is None else mv[1])
    r = gs.Renderer(wl.scene.n, wl.scene.sh_degree, wl.cams, tile=tile or wl.tile,
                    foveated=fov is not None, backward=backward, max_pairs=max_pairs,
                    chunk=chunk, chunk_slots=chunk_slots, tight=tight, multi_model=multi_model)
    if max_pairs:
        r.project(sc, f)
        r.bin_sort()
    else:
        r.fit(sc, f)
    out = r.alloc_outputs(fov=fov is not None, stats=stats)
    r.render(out, bg=bg, fov=fov is not None)
    torch.cuda.synchronize()
    return r, out, sc, f


def compare_images(rgb_gpu, img, sel=None, label=""):
    """Compare GPU colours with the oracle image `img` (optionally at the
    oracle pixels `sel`).  Unambiguous pixels: max abs <= 1e-3 and mean abs
    <= 1e-5 per channel.  Decision-ambiguous pixels: within the oracle's
    bound on a flipped decision plus 1e-3.  Prints and returns
    (max_err_clear, mean_err, n_ambiguous)."""
    sel = np.arange(len(img.rgb)) if sel is None else sel
    diff = np.abs(rgb_gpu.astype(np.float64) - img.rgb[sel])
    err = diff.max(axis=1)
    amb = img.amb[sel]
    clear = ~amb
    max_clear = float(err[clear].max()) if clear.any() else 0.0
    mean_err = float(diff[clear].mean()) if clear.any() else 0.0
    print(f"[parity{(' ' + label) if label else ''}] pixels {len(sel)}: max abs {max_clear:.3g}, "
          f"mean abs {mean_err:.3g}, decision-ambiguous {int(amb.sum())} "
          f"(max err {float(err[amb].max()) if amb.any() else 0.0:.3g})")
    assert max_clear <= IMG_MAX_ABS, f"max abs error {max_clear:.3g} on unambiguous pixels"
    assert mean_err <= IMG_MEAN_ABS, f"mean abs error {mean_err:.3g}"
    if amb.any():
        bound = img.ambB[sel][amb] + IMG_MAX_ABS
        assert np.all(err[amb] <= bound), "ambiguous pixel beyond its bound"
    assert amb.mean() <= AMBIG_MAX_FRACTION, f"{int(amb.sum())} decision-ambiguous pixels"
    return max_clear, mean_err, int(amb.sum())


# Gradients (backward vs the FP64 oracle's analytic gradient).
GRAD_REL = 1e-3
# Absolute part of the per-element bound: a finite-precision gradient errs
# by its relative rounding times the magnitude of the terms the element sums,
# however much they cancel.  The oracle returns that magnitude (the chain with
# every term in absolute value, `Grads.mag`); the CUDA path's terms carry
# FP32 values of relative error ~1e-6 (conic, mean, alpha, T) and sums over
# up to ~10^2 partial sums (warp reductions, atomics): 1e-5 of the magnitude,
# with a margin.  Without magnitudes (older callers) the bound falls back to
# 1e-4 of the point's row maximum + 1e-5 of the group maximum.
MAG_EPS = 1e-5
ROW_EPS = 1e-4
GROUP_EPS = 1e-5


def compare_grads(name, got, ref, mag=None):
    """Element by element: |g - r| <= 1e-3 |r| + 1e-5 mag (mag: sum of |term|
    behind the element, from the oracle), else 1e-3 |r| + 1e-4 max|r_row| +
    1e-5 max|r| with a row = one point's components in this group."""
    n = ref.shape[0]
    got = np.asarray(got, np.float64).reshape(n, -1)
    ref = np.asarray(ref, np.float64).reshape(n, -1)
    gmax = np.abs(ref).max() if ref.size else 0.0
    if gmax == 0:
        assert np.abs(got).max() < 1e-6, name
        return 0.0
    row = np.abs(ref).max(axis=1, keepdims=True)
    if mag is not None:
        mag = np.asarray(mag, np.float64).reshape(n, -1)
        tol = GRAD_REL * np.abs(ref) + MAG_EPS * mag + 1e-9 * gmax
        rule = f"1e-3 |r| + {MAG_EPS} sum|terms|"
    else:
        tol = GRAD_REL * np.abs(ref) + ROW_EPS * row + GROUP_EPS * gmax
        rule = f"1e-3 |r| + {ROW_EPS} row max + {GROUP_EPS} group max"
    err = np.abs(got - ref)
    ratio = err / tol
    worst = np.unravel_index(np.argmax(ratio), ratio.shape)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    extra = ""
    if mag is not None:
        em = err / np.maximum(mag, 1e-300)
        extra = f"; max err/sum|terms| {em.max():.3g}"
    print(f"[grad {name}] elements {ref.size}: worst err/tol {ratio.max():.3g} at {worst} "
          f"(got {got[worst]:.6g}, ref {ref[worst]:.6g}); 2-norm rel {rel:.3g}{extra}")
    if not np.all(err <= tol):
        for i, j in np.argwhere(err > tol)[:5]:
            print(f"  beyond: [{i},{j}] got {got[i, j]:.6g} ref {ref[i, j]:.6g} row max "
                  f"{row[i, 0]:.3g} group max {gmax:.3g} tol {tol[i, j]:.3g}"
                  + (f" sum|terms| {mag[i, j]:.3g}" if mag is not None else ""))
    assert np.all(err <= tol), f"{name}: {int((err > tol).sum())} elements beyond {rule}"
    return rel
