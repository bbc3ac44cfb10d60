"""Autotuner of the plan options that change speed but not results.

For a given scene, set of views and foveation it times complete frames
(projection, binning and sorting, rendering) for each candidate option set
(a list, or a coordinate search over the options) and returns the fastest.
Options: tile edge (16 or 8 pixels), digit width of the pair sort's radix
passes, and the heavy-tile chunk length.  Images do
not depend on these options (up to float rounding of the chunk merge), so the
choice is free.  Results can be cached in a JSON file keyed by the workload's
shape.

Candidates that do not fit (for example more tile/point pairs than 32-bit
indices address with 8x8 tiles) are skipped.
"""
from __future__ import annotations

import json
import os
import time

import torch

from .gs import GsError, Renderer

DEFAULT_CANDIDATES = [
    {"tile": 16, "radix_bits": 0, "chunk": 0},
    {"tile": 16, "radix_bits": 7, "chunk": 0},
    {"tile": 16, "radix_bits": 0, "chunk": 1024},
    {"tile": 16, "radix_bits": 0, "chunk": 2048},
    {"tile": 8, "radix_bits": 0, "chunk": 0},
    {"tile": 8, "radix_bits": 0, "chunk": 512},
]


def workload_key(n, sh_degree, cams, fov, tight=False) -> str:
    sizes = ",".join(f"{int(c[16])}x{int(c[17])}" for c in cams)
    return f"n={n};deg={sh_degree};fov={int(fov is not None)};tight={int(tight)};views={sizes}"


def _time_frames(r: Renderer, sc, fov, frames, warmup):
    out = r.alloc_outputs(fov=fov is not None)

    def frame():
        r.project(sc, fov)
        r.bin_sort()
        r.render(out, fov=fov is not None)

    for _ in range(warmup):
        frame()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(frames):
        frame()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / frames


# The search space of the coordinate search: each option's values, the
# first one the starting point.
SEARCH_SPACE = {"tile": [16, 8], "radix_bits": [0, 5, 6, 7, 8, 9, 10], "chunk": [0, 512, 1024, 2048, 4096]}


def autotune(sc: dict, n: int, sh_degree: int, cams, fov: dict | None = None,
             candidates=None, frames: int = 3, warmup: int = 1, cache_path: str | None = None,
             headroom: float = 1.05, tight: bool = False, verbose: bool = False,
             search: str = "list", space: dict | None = None, sweeps: int = 2) -> dict:
    """Return {"options": best option dict, "ms": its frame time, "trials": [...]}.

    search="list" times every candidate (``candidates`` or the defaults);
    search="coordinate" walks the search space one option at a time (tile
    edge, then digit width, then chunk length), keeping the best value of each
    before moving to the next, for up to ``sweeps`` sweeps or until a sweep
    improves nothing; every configuration is timed once."""
    key = workload_key(n, sh_degree, cams, fov, tight) + f";search={search}"
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return cache[key]
    trials = []
    seen = {}

    def trial(opt):
        k = (opt["tile"], opt["radix_bits"], opt["chunk"])
        if k in seen:
            return seen[k]
        t0 = time.perf_counter()
        r = None
        try:
            r = Renderer(n, sh_degree, cams, tile=opt["tile"], foveated=fov is not None,
                         radix_bits=opt["radix_bits"], chunk=opt["chunk"], tight=tight)
            r.fit(sc, fov, headroom=headroom)
            ms = _time_frames(r, sc, fov, frames, warmup)
            trials.append({**opt, "ms": round(ms, 4)})
        except (GsError, RuntimeError, torch.cuda.OutOfMemoryError) as e:
            trials.append({**opt, "ms": None, "error": str(e)[:120]})
        finally:
            r = None
            torch.cuda.empty_cache()
        if verbose:
            print(trials[-1], f"({time.perf_counter() - t0:.1f} s)")
        seen[k] = trials[-1]["ms"]
        return seen[k]

    if search == "coordinate":
        sp = space or SEARCH_SPACE
        cur = {k: v[0] for k, v in sp.items()}
        best_ms = trial(cur)
        for _ in range(sweeps):
            improved = False
            for name, values in sp.items():
                for v in values:
                    cand = {**cur, name: v}
                    ms = trial(cand)
                    if ms is not None and (best_ms is None or ms < best_ms):
                        best_ms, cur, improved = ms, cand, True
            if not improved:
                break
    else:
        for opt in candidates or DEFAULT_CANDIDATES:
            trial(opt)
    ok = [t for t in trials if t["ms"] is not None]
    if not ok:
        raise RuntimeError(f"no candidate fits: {trials}")
    best = min(ok, key=lambda t: t["ms"])
    res = {"options": {k: best[k] for k in ("tile", "radix_bits", "chunk")}, "ms": best["ms"],
           "trials": trials}
    if cache_path:
        cache = {}
        if os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
        cache[key] = res
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return res
