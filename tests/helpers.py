"""Shared helpers of the GPU tests: run the CUDA path and the oracle on the
same seeded inputs and compare."""
import numpy as np

# Image tolerance of the forward path (per RGB channel, colours in [0, 1]).
IMG_MAX_ABS = 1e-3
IMG_MEAN_ABS = 1e-5
# A pixel whose alpha-floor or early-stop decision lies within this relative
# distance of its threshold may legitimately take the other branch in FP32;
# it is compared against a looser bound (see ambiguous_bound).
AMBIG_MARGIN = 1e-4


# Ambiguous pixels must stay a small minority of the compared pixels.
AMBIG_MAX_FRACTION = 0.02


def ambiguous_bound(img, sel):
    """A flipped alpha-floor or stop decision at transmittance T changes the
    pixel by at most T times (the point's colour plus what follows), below
    T times twice the largest colour; colours of these scenes stay below 1.5."""
    return 3.0 * img.ambT[sel] + IMG_MAX_ABS


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


def compare_images(rgb_gpu, img, sel=None):
    """Compare GPU colours with the oracle image `img` (optionally at the
    oracle pixels `sel`).  Unambiguous pixels: max abs <= 1e-3 and mean abs
    <= 1e-5 per channel.  Decision-ambiguous pixels: within the bound that a
    flipped decision allows.  Returns (max_err_clear, mean_err, n_ambiguous)."""
    sel = np.arange(len(img.rgb)) if sel is None else sel
    diff = np.abs(rgb_gpu.astype(np.float64) - img.rgb[sel])
    err = diff.max(axis=1)
    amb = img.margin[sel] < AMBIG_MARGIN
    clear = ~amb
    max_clear = float(err[clear].max()) if clear.any() else 0.0
    mean_err = float(diff[clear].mean()) if clear.any() else 0.0
    assert max_clear <= IMG_MAX_ABS, f"max abs error {max_clear:.3g} on unambiguous pixels"
    assert mean_err <= IMG_MEAN_ABS, f"mean abs error {mean_err:.3g}"
    if amb.any():
        bound = ambiguous_bound(img, sel[amb])
        assert np.all(err[amb] <= bound), "ambiguous pixel beyond its bound"
    assert amb.mean() <= AMBIG_MAX_FRACTION, f"{int(amb.sum())} decision-ambiguous pixels"
    return max_clear, mean_err, int(amb.sum())
