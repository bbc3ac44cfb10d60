"""Benchmark of the GB300 tile rasterizer.

Headline (``value``): frames/s of the plain forward path (projection, tile
binning + radix sorts, rasterization) on the 1920x1080, 1M-point, SH degree 3
blob workload, inputs resident in HBM.  Each step renders one frame.  One
JSON line on stdout (rank 0).

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload (the paper ships no code; the oracle is the reference arm).
Under torchrun every rank renders its own replica of the workload (views are
independent: no collective); ``value`` sums the ranks' frames.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FPS & Gpix/s @1080p, 1M Gaussians: batched/foveated vs plain; bwd ms/view"
L2_FLUSH_BYTES = 256 << 20     # > 129 MB L2
# the headline workload, the same for both arms
HEADLINE_CONFIG = {"workload": "plain_1920x1080_n1M_sh3", "points": 1_000_000, "sh_degree": 3,
                   "resolution": "1920x1080", "tile": 16, "views_per_step": 1,
                   "support": "tight: tiles of the 3-sigma rectangle that the alpha >= 1/255 "
                              "ellipse reaches (same image)"}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="headline only")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    ap.add_argument("--only", nargs="*", default=None, help="extras to run")
    ap.add_argument("--batch-views", type=int, default=None,
                    help="64-view batch extra: first N views only (profiling a smaller case)")
    ap.add_argument("--batch-points", type=int, default=None,
                    help="64-view batch extra: N points instead of 6M (profiling a smaller case)")
    ap.add_argument("--no-separate-plans", action="store_true",
                    help="64-view batch extra: skip the separate single-view plans")
    ap.add_argument("--batch-options", default=None,
                    help="64-view batch extra: tile,radix_bits,chunk instead of the autotuner")
    ap.add_argument("--fov-points", type=int, default=None,
                    help="foveated stereo extra: N points instead of 3M (profiling a smaller case)")
    ap.add_argument("--fwdbwd-views", type=int, default=None,
                    help="forward+backward extra: first N views only (profiling a smaller case)")
    return ap.parse_args(argv)


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# FP32 ALU issue peak: SMs x 128 FP32 lanes per clock (the SM count is the
# device's own, cudaDevAttrMultiProcessorCount).
FP32_LANES = 128
# Algorithmic FP32 operations of the render inner loop: per (pixel, point)
# evaluation the whitened quadratic form and the floor test (2 sub, 2 mul +
# 2 fma for t1/t2, 1 mul + 1 fma for |t|^2, 1 add of log2 o, 1 compare = 10);
# per blend the clamp, 1 - alpha, T update, stop test, weight and 3 colour
# fma (8) plus one ex2 on the SFU.
OPS_PER_EVAL = 10
OPS_PER_BLEND = 8


RENDER_SOURCES = ("paper_2407_00435_gb300/csrc/k_render.cu", "paper_2407_00435_gb300/csrc/raster.cuh")
# DRAM bytes per launch of the headline render kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), with the hash of the
# kernel's sources at capture time; the summary beside it gives the command.
RENDER_TRAFFIC = "profiles/render_plain_1080p_n1M.json"


def depth_passes(r, gs):
    """Depth-sort passes of the plan's last frame: with the cooperative sort,
    9-bit digits over the span of the visible depth keys; else four."""
    if not gs._lib.gs_sort_is_cooperative():
        return 4
    import torch
    d = r.region(gs.GS_REGION_ITEM_DEPTH, torch.int32, r.n * r.V)
    d = d.to(torch.int64) & 0xffffffff
    vis = d[d != 0xffffffff]
    if vis.numel() == 0:
        return 1
    span = int(vis.max() - vis.min())
    return max(1, (max(span, 1).bit_length() + 8) // 9)


def bin_sort_bytes(n_slots, m_visible, k_pairs, tiles, pair_passes, tight, fov, depth_passes=4):
    """Algorithmic DRAM bytes of one gs_bin_sort (the kernels' own minimal
    reads and writes, no cache effects):
      pair count   per item slot: depth key 4 read; per visible item:
                   rectangle 8 (+ tight support 24) read, count 4 + emit
                   record 16 (+ row table 16 with a filter) + count word 4
                   written
      depth sort   pass 0 over every slot: count read 4 + key read 4, the
                   visible items' key and value written 8 (invisible slots
                   are dropped); each later pass per visible item: count
                   read 4, key + value read 8 and written 8
      offsets      per visible item: item 4 read, count word 4 gathered,
                   count 4 written in depth order; count 4 read, offset 4
                   written
      emit         per visible item: item 4 + offset 4 + count 4 read, emit
                   record 16 (+ 16 row table) gathered; per pair 8 written
      pair sort    per pair and pass: count read 4, key + value read 8 and
                   written 8
      ranges       per pair 4 read; per tile 8 written (+ 8 cleared)"""
    table = 16 if (tight or fov) else 0
    count = n_slots * 4 + m_visible * (8 + (24 if tight else 0) + 4 + 16 + table + 4)
    depth = n_slots * 8 + m_visible * 8 + (depth_passes - 1) * m_visible * 20
    offsets = m_visible * (4 + 4 + 4 + 4 + 4)
    emit = m_visible * (4 + 4 + 4 + 16 + table) + 8 * k_pairs
    pair = pair_passes * 20 * k_pairs
    ranges = 4 * k_pairs + 16 * tiles
    return count + depth + offsets + emit + pair + ranges


def pair_passes(tiles, radix_bits=0):
    bits = max(1, int(tiles - 1).bit_length())
    want = radix_bits or 8
    return min(4, (bits + want - 1) // want)


def max_over_ranks(torch, dist, x, world, device):
    """The largest of the ranks' values of x (a job's step time is its
    slowest rank's); x itself with one rank."""
    if world <= 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ms_max, world):
    """Whole-job frames/s of `world` replicas whose slowest takes ms_max per frame."""
    return 1000.0 / ms_max * world


def peak_probe(torch, gs, iters=20000, reps=5):
    """Measured FP32 FMA and ex2 lane-op rates (T ops/s): best of `reps`
    event-timed launches of the library's probe kernel."""
    sink = torch.zeros(1, device="cuda")
    out = []
    for kind in (0, 1):
        gs.gs_peak_probe(kind, 100, sink)
        best = None
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            ops = gs.gs_peak_probe(kind, iters, sink)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        out.append(round(ops / (best * 1e-3) / 1e12, 3))
    return out


def render_sources_sha1():
    import hashlib
    h = hashlib.sha1()
    for f in RENDER_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def captured_traffic():
    """DRAM bytes per launch of the render kernel from the committed capture
    record, or None when the kernel's sources changed since the capture."""
    try:
        with open(os.path.join(ROOT, RENDER_TRAFFIC)) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None, None
    if rec.get("kernel_source_sha1") != render_sources_sha1():
        return None, rec.get("kernel_source_sha1")
    try:
        return int(rec["dram_bytes_per_launch"]), rec["kernel_source_sha1"]
    except (KeyError, ValueError, TypeError):
        return None, None


def host_info():
    """Host cores and CPU model (the CPU baseline's machine)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k = ln.split(":", 1)[0].strip().lower()
                if k in ("model name", "cpu model", "hardware"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "cpu_model": model}


class L2Flusher:
    def __init__(self, torch):
        self.buf = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def __call__(self):
        self.buf.fill_(1)


def time_steps(torch, fn, steps, warmup, flush, inner=None):
    """Time `steps` calls of fn() with CUDA events on the current stream,
    flushing L2 between steps (outside the event pairs).  If `inner` is a
    list, fn(inner_events) may record per-kernel event pairs into it."""
    for _ in range(warmup):
        fn(None)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    evs = []
    kev = []
    for _ in range(steps):
        flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        fn(kev)
        b.record(st)
        evs.append((a, b))
    torch.cuda.synchronize()
    total = sum(a.elapsed_time(b) for a, b in evs)
    k_ms = [a.elapsed_time(b) for a, b in kev]
    return total, k_ms


def gpu_arm(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2407_00435_gb300 import gs, synth
    from paper_2407_00435_gb300.pipeline import HostFramePipeline

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    flush = L2Flusher(torch)

    # ---- headline: plain forward, 1080p, 1M points, SH3 ---------------------
    wl = synth.workload(1)
    assert wl.name == HEADLINE_CONFIG["workload"] and wl.scene.n == HEADLINE_CONFIG["points"]
    sc = gs.scene_to_device(wl.scene)
    r = gs.Renderer(wl.scene.n, wl.scene.sh_degree, wl.cams, tight=True)
    c = r.fit(sc)
    out = r.alloc_outputs(stats=True)
    r.render(out)                                   # untimed: exact counts
    code, cnt = r.counters()
    assert code == gs.GS_OK, cnt
    n_evals, n_blends = int(cnt["n_evals"]), int(cnt["n_blends"])
    out = r.alloc_outputs()

    stage_ev = []

    def step(kev):
        if kev is None:
            r.project(sc)
            r.bin_sort()
            r.render(out)
            return
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record()
        r.project(sc)
        e[1].record()
        r.bin_sort()
        e[2].record()
        r.render(out)
        e[3].record()
        kev.append((e[2], e[3]))
        stage_ev.append(e)

    for _ in range(args.warmup):
        step(None)
    torch.cuda.synchronize()
    # the frame as one CUDA graph (the library's launches are capturable):
    # the timed steps replay it
    cap = torch.cuda.Stream()
    cap.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(cap):
        step(None)
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=cap):
            step(None)
    torch.cuda.current_stream().wait_stream(cap)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        total_ms, _ = time_steps(torch, lambda kev: graph.replay(), args.steps, 0, flush)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    code, cnt2 = r.counters()
    assert code == gs.GS_OK, cnt2
    ms = max_over_ranks(torch, dist, total_ms / args.steps, world, "cuda")
    value = job_rate(ms, world)
    clocks = clk.summary()
    # the stages (and the render kernel alone) timed apart, with events
    # between them, on stream-launched frames
    _, k_ms = time_steps(torch, step, max(5, args.steps // 2), 0, flush)
    render_ms = sorted(k_ms)[len(k_ms) // 2]
    stages = {nm: round(sorted(e[q].elapsed_time(e[q + 1]) for e in stage_ev)[len(stage_ev) // 2], 4)
              for q, nm in enumerate(("project", "bin_sort", "render"))}

    # roofline of the dominant kernel (render): FP32 issue bound
    peaks, src = _peaks()
    mhz = peaks.get("sm_max_mhz", 2070.0)
    n_sm = int(torch.cuda.get_device_properties(local).multi_processor_count)
    peak_tops = n_sm * FP32_LANES * mhz * 1e6 / 1e12
    achieved_tops = (OPS_PER_EVAL * n_evals + OPS_PER_BLEND * n_blends) / (render_ms * 1e-3) / 1e12
    traffic, _ = captured_traffic()
    probe = peak_probe(torch, gs)
    roofline = {"bound": "alu", "kernel": "k_render", "achieved": round(achieved_tops, 3),
                "peak": round(peak_tops, 3), "unit": "TFLOP/s (FP32 lane-ops)",
                "frac": round(achieved_tops / peak_tops, 4), "traffic": traffic,
                "traffic_source": RENDER_TRAFFIC if traffic else None,
                "sm_count": n_sm,
                "peak_source": f"{n_sm} SMs (device attribute) x {FP32_LANES} FP32 lanes x "
                               f"{mhz:.0f} MHz ({src} sm_max_mhz); of measured",
                "render_ms": round(render_ms, 4),
                "probe": {"fma_tops": probe[0], "ex2_tops": probe[1],
                          "frac_of_fma_probe": round(achieved_tops / probe[0], 4) if probe[0] else None,
                          "note": "measured issue rates of independent FP32 FMA / ex2 chains on "
                                  "every SM (gs_peak_probe), at the clock of the run"}}
    # the binning and sorting stage (pair count, depth sort, offsets, emit,
    # pair sort, ranges): HBM bound by design, algorithmic bytes / stage time
    bs_bytes = bin_sort_bytes(r.n * r.V, int(c["n_visible"]), int(c["n_pairs"]), r.T_tiles,
                              pair_passes(r.T_tiles), True, False, depth_passes(r, gs))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    bs_gbs = bs_bytes / (stages["bin_sort"] * 1e-3) / 1e9
    roofline_bin_sort = {"bound": "hbm", "stage": "gs_bin_sort", "achieved": round(bs_gbs, 1),
                         "peak": hbm, "unit": "GB/s", "frac": round(bs_gbs / hbm, 4),
                         "bytes_per_frame": int(bs_bytes), "stage_ms": stages["bin_sort"],
                         "peak_source": f"{src} hbm_gbs (copy); of measured",
                         "note": "algorithmic bytes per kernel in bench.bin_sort_bytes; at this "
                                 "size much of the stage's working set is served from the "
                                 "129 MB L2"}

    # ---- end to end through the public API with host buffers ----------------
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(wl.scene, k2))).pin_memory()
            for k, k2 in (("means", "means"), ("scales", "scales"), ("quats", "quats"),
                          ("opac", "opac"), ("sh", "sh"))}
    rgb_host = [torch.empty(r.P, 3).pin_memory() for _ in range(2)]
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = rgb_host[0].numel() * 4
    # every frame uploads the whole scene from pinned host memory and reads its
    # image back; the upload of frame i+1 and the read-back of frame i - 1
    # overlap frame i's compute (HostFramePipeline); the scene (236 MB) is
    # larger than L2, so no flush between frames
    pipe = HostFramePipeline(r)
    k_e2e = max(8, args.steps)
    frames = [(host, rgb_host[i % 2]) for i in range(k_e2e)]
    pipe.run(frames[:args.warmup])
    torch.cuda.synchronize()
    ea = torch.cuda.Event(enable_timing=True)
    eb = torch.cuda.Event(enable_timing=True)
    pipe.run(frames, ea, eb)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(torch, dist, ea.elapsed_time(eb) / k_e2e, world, "cuda")
    code, cnt3 = r.counters()
    assert code == gs.GS_OK, cnt3
    gpu_launches = args.steps * r.launches_per_frame()

    P_head = r.P
    extras = {}
    if not args.no_extras:
        del r, host, out, pipe, frames
        torch.cuda.empty_cache()
        # the same frame with the plain 3-sigma rectangle support, for reference
        rr = gs.Renderer(wl.scene.n, wl.scene.sh_degree, wl.cams)
        cr = rr.fit(sc)
        outr = rr.alloc_outputs()

        def rect_frame():
            rr.project(sc)
            rr.bin_sort()
            rr.render(outr)

        ms_rect = _ms(torch, rect_frame, max(3, min(args.steps, 10)), 2, flush)
        extras["rect_support"] = {"fps": round(1000.0 / ms_rect, 2),
                                  "pairs_K": int(cr["n_pairs"]),
                                  "tight_speedup": round(ms_rect / ms, 3)}
        del rr, outr, sc
        torch.cuda.empty_cache()
        steps_x = max(3, min(args.steps, 10))
        for name, fn in (("foveated_stereo", extra_foveated),
                         ("foveated_ce_levels", extra_foveated_ce), ("multi_model_fr", extra_mmfr),
                         ("fwd_bwd", extra_fwd_bwd), ("hvsq", extra_hvsq),
                         ("prune_round", extra_prune), ("batched_64_views", extra_batched)):
            if args.only and name not in args.only:
                continue
            try:
                if name == "batched_64_views":
                    extras[name] = fn(torch, gs, synth, flush, steps_x, args.batch_views,
                                      args.batch_points, not args.no_separate_plans,
                                      args.batch_options)
                elif name == "foveated_stereo":
                    extras[name] = fn(torch, gs, synth, flush, steps_x, args.fov_points)
                elif name == "fwd_bwd":
                    extras[name] = fn(torch, gs, synth, flush, steps_x, args.fwdbwd_views)
                else:
                    extras[name] = fn(torch, gs, synth, flush, steps_x)
            except Exception as e:  # report, never hide
                extras[name] = {"error": f"{type(e).__name__}: {e}"}
    res = {
        "metric": METRIC, "value": round(value, 2), "unit": "frames/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded blob-mixture scene; the paper's datasets are not available)",
        "config": {**HEADLINE_CONFIG,
                   "pairs_K": int(c["n_pairs"]), "visible": int(c["n_visible"]),
                   "l2": "flushed between steps (256 MB write) and scene 236 MB > L2",
                   "timing": "each step replays the frame (projection, binning and sorting, "
                             "render) captured as one CUDA graph",
                   "parallelism": f"replicas x{world}"},
        "gpix_per_s": round(value * P_head / 1e9, 3),
        "blends_per_s": round(n_blends * value, 1),
        "evals_per_s": round(n_evals * value, 1),
        "stages_ms": stages,
        "roofline": roofline,
        "roofline_bin_sort": roofline_bin_sort,
        "e2e": {"value": round(job_rate(e2e_ms, world), 2), "unit": "frames/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "pipelined": "scene upload of frame i+1 and image read-back of frame i-1 "
                             "overlap frame i (copy, compute, read-back streams)"},
        "clocks": clocks,
        "gpu_launches": gpu_launches,
        "extras": extras,
    }
    return res, rank, world


# --------------------------------------------------------------------------
# the other workloads: foveated stereo, forward+backward, batched views
# --------------------------------------------------------------------------
def _ms(torch, fn, steps, warmup, flush):
    total, _ = time_steps(torch, lambda kev: fn(), steps, warmup, flush)
    return total / steps


def extra_foveated(torch, gs, synth, flush, steps, points=None):
    """3M points, 2 eyes at 1920x1920, 4 nested levels: foveated vs plain."""
    wl = synth.workload(2, n=points)
    sc = gs.scene_to_device(wl.scene)
    f = gs.fov_to_device(wl.fov)
    rf = gs.Renderer(wl.scene.n, 3, wl.cams, foveated=True, tight=True)
    cf = rf.fit(sc, f)
    of = rf.alloc_outputs(fov=True, stats=True)
    rf.render(of, fov=True)
    _, cntf = rf.counters()
    of = rf.alloc_outputs(fov=True)
    rp = gs.Renderer(wl.scene.n, 3, wl.cams, tight=True)
    cp = rp.fit(sc)
    op = rp.alloc_outputs(stats=True)
    rp.render(op)
    _, cntp = rp.counters()
    op = rp.alloc_outputs()

    def fov_step():
        rf.project(sc, f)
        rf.bin_sort()
        rf.render(of, fov=True)

    def plain_step():
        rp.project(sc)
        rp.bin_sort()
        rp.render(op)

    ms_f = _ms(torch, fov_step, steps, 2, flush)
    ms_p = _ms(torch, plain_step, steps, 2, flush)
    px = rf.P
    # the foveated frame's stages, timed apart, and the foveated render's
    # roofline (the plain render's op count per walked position and blend)
    st = {"project": [], "bin_sort": [], "render": []}
    for _ in range(max(3, steps // 2)):
        flush()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record()
        rf.project(sc, f)
        ev[1].record()
        rf.bin_sort()
        ev[2].record()
        rf.render(of, fov=True)
        ev[3].record()
        torch.cuda.synchronize()
        for q, nm in enumerate(("project", "bin_sort", "render")):
            st[nm].append(ev[q].elapsed_time(ev[q + 1]))
    stages = {k: round(sorted(v)[len(v) // 2], 4) for k, v in st.items()}
    # one more staged frame in an NVTX range (what kernel profiles of this
    # workload select)
    flush()
    torch.cuda.nvtx.range_push("foveated_frame")
    rf.project(sc, f)
    rf.bin_sort()
    rf.render(of, fov=True)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    peaks, _ = _peaks()
    n_sm = int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)
    peak_tops = n_sm * FP32_LANES * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    ach = (OPS_PER_EVAL * int(cntf["n_evals"]) + OPS_PER_BLEND * int(cntf["n_blends"])) / \
        (stages["render"] * 1e-3) / 1e12
    del rf, rp, sc
    torch.cuda.empty_cache()
    return {"workload": wl.name, "fps_foveated": round(1000 / ms_f, 2),
            "stages_ms_foveated": stages,
            "roofline_render_foveated": {"bound": "alu", "achieved": round(ach, 3),
                                         "peak": round(peak_tops, 3),
                                         "unit": "TFLOP/s (FP32 lane-ops)",
                                         "frac": round(ach / peak_tops, 4),
                                         "note": "both eyes' render, ops as the plain render's "
                                                 "roofline; of measured"},
            "fps_plain": round(1000 / ms_p, 2), "speedup": round(ms_p / ms_f, 3),
            "gpix_per_s_foveated": round(px / ms_f / 1e6, 3),
            "pairs_foveated": int(cf["n_pairs"]), "pairs_plain": int(cp["n_pairs"]),
            "blends_per_s_foveated": round(int(cntf["n_blends"]) * 1000 / ms_f, 1),
            "per_pixel": {"walked_foveated": round(int(cntf["n_evals"]) / px, 1),
                          "blended_foveated": round(int(cntf["n_blends"]) / px, 1),
                          "walked_plain": round(int(cntp["n_evals"]) / px, 1),
                          "blended_plain": round(int(cntp["n_blends"]) / px, 1)},
            "frame": "2 eyes"}


def extra_foveated_ce(torch, gs, synth, flush, steps):
    """The foveated stereo frame with its nested levels built as the paper
    builds them (Sec. 3.4, 4.2): each coarser level keeps the points of the
    finer one with the highest computational efficiency (CE maximum over the
    two eye poses and two orbit poses, from the render's statistics; the
    library's stable mask), in the proportions of the random levels (N, N/2,
    N/4, N/8).  Compared with the random levels of the same scene."""
    import numpy as np
    wl = synth.workload(2)
    n = wl.scene.n
    sc = gs.scene_to_device(wl.scene)
    rng = np.random.default_rng(2025)
    poses = np.concatenate([wl.cams, synth.orbit_cameras(rng, 2, 4.0, [(1920, 1920)] * 2)])
    ce = torch.zeros(n, device="cuda")
    last = None
    for v in range(len(poses)):
        rv = gs.Renderer(n, 3, poses[v:v + 1], tight=True)
        rv.fit(sc, headroom=1.05)
        o = rv.alloc_outputs(stats=True)
        rv.render(o)
        gs.gs_ce_update(n, o["stats"], ce)
        if last is not None:
            del last
        last = rv
    m = torch.ones(n, dtype=torch.uint8, device="cuda")
    for frac in (0.5, 0.75, 0.875):          # levels 2, 3, 4 keep 1/2, 1/4, 1/8
        m += last.prune_mask(ce, frac)
    del last
    torch.cuda.empty_cache()
    res = {"workload": wl.name, "levels": "CE-ranked nested subsets (N, N/2, N/4, N/8)"}
    for name, bound in (("ce_levels", m), ("random_levels", None)):
        f = gs.fov_to_device(wl.fov)
        if bound is not None:
            f["bound_m"] = bound
        r = gs.Renderer(n, 3, wl.cams, foveated=True, tight=True)
        c = r.fit(sc, f)
        o = r.alloc_outputs(fov=True, stats=True)
        r.render(o, fov=True)
        _, cnt = r.counters()
        out = r.alloc_outputs(fov=True)

        def step():
            r.project(sc, f)
            r.bin_sort()
            r.render(out, fov=True)

        ms = _ms(torch, step, steps, 2, flush)
        res[name] = {"fps": round(1000.0 / ms, 2), "pairs": int(c["n_pairs"]),
                     "walked_per_pixel": round(int(cnt["n_evals"]) / r.P, 1),
                     "blended_per_pixel": round(int(cnt["n_blends"]) / r.P, 1)}
        del r, o, out
        torch.cuda.empty_cache()
    del sc
    torch.cuda.empty_cache()
    return res


def extra_mmfr(torch, gs, synth, flush, steps):
    """The foveated stereo frame with a separate model per level (the
    multi-model pipeline of Sec. 4.1; level-l model = its own copy of the
    nested level-l subset, 1.875 x 3M points) against the nested-subset
    representation of the same levels."""
    wl = synth.multi_model_workload()
    sc = gs.scene_to_device(wl.scene)
    f = gs.fov_to_device(wl.fov)
    r = gs.Renderer(wl.scene.n, 3, wl.cams, multi_model=True, tight=True)
    c = r.fit(sc, f)
    out = r.alloc_outputs(fov=True)

    def step():
        r.project(sc, f)
        r.bin_sort()
        r.render(out, fov=True)

    ms = _ms(torch, step, steps, 2, flush)
    res = {"workload": wl.name, "points": wl.scene.n, "fps_multi_model": round(1000 / ms, 2),
           "pairs_multi_model": int(c["n_pairs"])}
    del r, out, sc, f
    torch.cuda.empty_cache()
    wn = synth.workload(2)
    sc = gs.scene_to_device(wn.scene)
    f = gs.fov_to_device(wn.fov)
    r = gs.Renderer(wn.scene.n, 3, wn.cams, foveated=True, tight=True)
    c = r.fit(sc, f)
    out = r.alloc_outputs(fov=True)

    def step_n():
        r.project(sc, f)
        r.bin_sort()
        r.render(out, fov=True)

    ms_n = _ms(torch, step_n, steps, 2, flush)
    res.update({"fps_nested": round(1000 / ms_n, 2), "pairs_nested": int(c["n_pairs"]),
                "nested_speedup": round(ms / ms_n, 3), "frame": "2 eyes"})
    del r, out, sc, f
    torch.cuda.empty_cache()
    return res


def extra_fwd_bwd(torch, gs, synth, flush, steps, views=None):
    """500k points, SH3, 8 views at 1024^2, L1 loss, forward + backward:
    the views foveated in one batched plan (4 nested levels, rings at
    10/20/35 degrees, 32-px band: retraining through the foveated renderer,
    Sec. 4.3) against 8 plain per-view plans, and the plain batched plan."""
    import numpy as np
    from paper_2407_00435_gb300 import autograd as ga
    wl = synth.workload(3, views=views)
    wf = synth.fov_fwd_bwd_workload(views=views)
    sc = gs.scene_to_device(wl.scene)
    f = gs.fov_to_device(wf.fov)
    V = len(wl.cams)
    rng = np.random.default_rng(1003)
    target = torch.from_numpy(rng.uniform(0, 1, (V * 1024 * 1024, 3)).astype(np.float32)).cuda()
    rb = gs.Renderer(wl.scene.n, 3, wl.cams, backward=True, tight=True)
    rb.fit(sc)
    rf = gs.Renderer(wl.scene.n, 3, wf.cams, foveated=True, backward=True, tight=True)
    cf = rf.fit(sc, f)
    per = [gs.Renderer(wl.scene.n, 3, wl.cams[v:v + 1], backward=True, tight=True)
           for v in range(V)]
    for r in per:
        r.fit(sc)
    g = {k: torch.empty_like(v) for k, v in sc.items()}
    ob = rb.alloc_outputs()
    of = rf.alloc_outputs(fov=True)
    ov = [r.alloc_outputs() for r in per]
    npx = 1024 * 1024

    def batched():
        rb.project(sc)
        rb.bin_sort()
        rb.render(ob)
        dL = torch.sign(ob["rgb"] - target) / ob["rgb"].numel()
        rb.backward(dL, ob, g)

    def batched_fov():
        rf.project(sc, f)
        rf.bin_sort()
        rf.render(of, fov=True)
        dL = torch.sign(of["rgb"] - target) / of["rgb"].numel()
        rf.backward(dL, of, g)

    def per_view():
        for v, r in enumerate(per):
            r.project(sc)
            r.bin_sort()
            r.render(ov[v])
            tv = target[v * npx:(v + 1) * npx]
            dL = torch.sign(ov[v]["rgb"] - tv) / (ov[v]["rgb"].numel() * V)
            r.backward(dL, ov[v], g)

    def bwd_only():
        dL = torch.sign(ob["rgb"] - target) / ob["rgb"].numel()
        rb.backward(dL, ob, g)

    def bwd_only_fov():
        dL = torch.sign(of["rgb"] - target) / of["rgb"].numel()
        rf.backward(dL, of, g)

    ms_b = _ms(torch, batched, steps, 2, flush)
    ms_f = _ms(torch, batched_fov, steps, 2, flush)
    ms_v = _ms(torch, per_view, steps, 2, flush)
    batched()
    ms_bwd = _ms(torch, bwd_only, steps, 2, flush)
    batched_fov()
    ms_bwd_f = _ms(torch, bwd_only_fov, steps, 2, flush)
    # autograd path (L1 loss through torch.autograd.Function)
    scg = {k: v.clone().requires_grad_(True) for k, v in sc.items()}

    def autograd_step():
        for v in scg.values():
            v.grad = None
        loss = ga.l1_loss(ga.render(scg, rb, check=False), target)
        loss.backward()

    ms_ag = _ms(torch, autograd_step, steps, 2, flush)
    pairs_plain = int(rb.counters()[1]["n_pairs"])
    del rb, rf, per, sc
    torch.cuda.empty_cache()
    return {"workload": wl.name, "views": V, "fwd_bwd_ms_batched": round(ms_b, 3),
            "fwd_bwd_ms_per_view_plans": round(ms_v, 3), "speedup": round(ms_v / ms_b, 3),
            "bwd_ms_per_view": round(ms_bwd / V, 4), "autograd_step_ms": round(ms_ag, 3),
            "foveated": {"workload": wf.name, "fwd_bwd_ms_batched_foveated": round(ms_f, 3),
                         "speedup_vs_plain_per_view_plans": round(ms_v / ms_f, 3),
                         "speedup_vs_plain_batched": round(ms_b / ms_f, 3),
                         "bwd_ms_per_view_foveated": round(ms_bwd_f / V, 4),
                         "pairs_foveated": int(cf["n_pairs"]), "pairs_plain": pairs_plain,
                         "note": "batched foveated forward+backward against plain per-view "
                                 "forward+backward of the same views; gradient parity of this "
                                 "plan at full size in tests/test_gpu_fullsize.py"}}


def extra_hvsq(torch, gs, synth, flush, steps):
    """HVSQ per quality level (Sec. 2.2; the quality loss of level training,
    Sec. 4.3) of the foveated stereo frame against the plain render of the
    same scene, both eyes at 1920^2, and its gradient: the loss a retraining
    step through the foveated renderer evaluates.  Pooling law r = floor(1 +
    0.025 e^2) px, regions = the frame's 4 levels (rings at 10/20/35 deg)."""
    import numpy as np
    wl = synth.workload(2)
    sc = gs.scene_to_device(wl.scene)
    f = gs.fov_to_device(wl.fov)
    rf = gs.Renderer(wl.scene.n, 3, wl.cams, foveated=True, tight=True)
    rf.fit(sc, f)
    of = rf.alloc_outputs(fov=True)
    rf.render(of, fov=True)
    rp = gs.Renderer(wl.scene.n, 3, wl.cams, tight=True)
    rp.fit(sc)
    op = rp.alloc_outputs()
    rp.render(op)
    pool_tan, r_base = synth.pooling_tangents()
    views = [gs.HvsqView(int(c[16]), int(c[17]), wl.fov.gaze[v], float(c[13]), wl.fov.ring_tan,
                         pool_tan, r_base) for v, c in enumerate(wl.cams)]
    npx = [v.W * v.H for v in views]
    out = [torch.empty(v.n_regions, dtype=torch.float64, device="cuda") for v in views]
    grad = torch.empty_like(of["rgb"])

    def step(with_grad):
        px = 0
        for v, o, n in zip(views, out, npx):
            v(of["rgb"][px:px + n], op["rgb"][px:px + n], o,
              grad[px:px + n] if with_grad else None)
            px += n

    ms_fb = _ms(torch, lambda: step(True), steps, 2, flush)
    ms_f = _ms(torch, lambda: step(False), steps, 2, flush)
    per_level = np.stack([o.cpu().numpy() for o in out])
    del rf, rp, sc, views
    torch.cuda.empty_cache()
    return {"workload": wl.name, "views": len(npx), "pixels": int(sum(npx)),
            "hvsq_fwd_bwd_ms": round(ms_fb, 3), "hvsq_fwd_ms": round(ms_f, 3),
            "gpix_per_s_fwd_bwd": round(sum(npx) / ms_fb / 1e6, 3),
            "hvsq_per_level_eye0": [float(x) for x in per_level[0]],
            "hvsq_per_level_eye1": [float(x) for x in per_level[1]],
            "pooling": "r = floor(1 + 0.025 e^2) px, e in degrees (at most 64)",
            "reference": "plain render of the same scene (altered: the foveated render)"}


def extra_prune(torch, gs, synth, flush, steps):
    """One round of efficiency-aware pruning (Sec. 3.2-3.4) on the 1080p/1M
    workload: statistics renders of 4 orbit poses + the bench pose, CE
    maximum over them, mask of the lowest 10%, stable compaction; then the
    frame rate and pair count of the pruned scene."""
    import numpy as np
    wl = synth.workload(1)
    sc = gs.scene_to_device(wl.scene)
    rng = np.random.default_rng(2024)
    poses = np.concatenate([wl.cams, synth.orbit_cameras(rng, 4, 4.0, [(1920, 1080)] * 4)])
    rs = [gs.Renderer(wl.scene.n, 3, poses[v:v + 1], tight=True) for v in range(len(poses))]
    for r in rs:
        r.fit(sc, headroom=1.05)
    outs = [r.alloc_outputs(stats=True) for r in rs]
    ce = torch.zeros(wl.scene.n, device="cuda")

    def prune_round():
        ce.zero_()
        for r, o in zip(rs, outs):
            r.project(sc)
            r.bin_sort()
            r.render(o)
            gs.gs_ce_update(wl.scene.n, o["stats"], ce)
        keep = rs[0].prune_mask(ce, 0.10)
        return rs[0].compact(sc, keep)

    pruned = prune_round()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    pruned = prune_round()
    t1.record()
    torch.cuda.synchronize()
    round_ms = t0.elapsed_time(t1)
    n_kept = int(pruned["means"].shape[0])
    res = {"workload": wl.name, "poses": len(poses), "fraction": 0.10,
           "points_before": wl.scene.n, "points_after": n_kept,
           "round_ms_incl_stats_renders": round(round_ms, 3)}
    for name, scene, n in (("before", sc, wl.scene.n), ("after", pruned, n_kept)):
        r = gs.Renderer(n, 3, wl.cams, tight=True)
        c = r.fit({k: v.contiguous() for k, v in scene.items()}, headroom=1.05)
        out = r.alloc_outputs()

        def frame():
            r.project({k: v.contiguous() for k, v in scene.items()})
            r.bin_sort()
            r.render(out)

        ms = _ms(torch, frame, steps, 2, flush)
        res[f"fps_{name}"] = round(1000.0 / ms, 2)
        res[f"pairs_{name}"] = int(c["n_pairs"])
        del r, out
    del rs, outs, sc, pruned
    torch.cuda.empty_cache()
    return res


def extra_batched(torch, gs, synth, flush, steps, views=None, points=None, separate=True,
                  options=None):
    """6M points, 64 views of uneven sizes, half foveated: project + sort +
    render of all views as one CUDA graph (one render launch for all tiles),
    with the plan options picked by the autotuner (a coordinate search over
    tile edge, pair-sort digit width and chunk length); the stages timed
    apart, the bin/sort stage against HBM, and the same views rendered as 64
    separate single-view plans."""
    import numpy as np
    from paper_2407_00435_gb300.autotune import autotune
    wl = synth.workload(4, n=points)
    if views:
        fv = wl.fov
        wl = synth.Workload(wl.name + f"_first{views}", wl.scene, wl.cams[:views], wl.tile,
                            synth.Foveation(fv.n_levels, fv.bound_m, fv.ring_tan, fv.band_px,
                                            fv.gaze[:views], fv.view_fov[:views]))
    sc = gs.scene_to_device(wl.scene)
    f = gs.fov_to_device(wl.fov)
    if options:
        t, rb, ch = (int(x) for x in options.split(","))
        tune = {"options": {"tile": t, "radix_bits": rb, "chunk": ch}, "trials": "given"}
    else:
        tune = autotune(sc, wl.scene.n, 3, wl.cams, f, frames=2, warmup=1, tight=True,
                        search="coordinate", sweeps=1)
    opt = tune["options"]
    r = gs.Renderer(wl.scene.n, 3, wl.cams, foveated=True, tight=True, tile=opt["tile"],
                    radix_bits=opt["radix_bits"], chunk=opt["chunk"])
    c = r.fit(sc, f, headroom=1.05)
    out = r.alloc_outputs(fov=True)

    def frame():
        r.project(sc, f)
        r.bin_sort()
        r.render(out, fov=True)

    frame()
    torch.cuda.synchronize()
    # stages, timed apart (outside the graph)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    st = {"project": [], "bin_sort": [], "render": []}
    for _ in range(max(2, steps // 2)):
        flush()
        ev[0].record()
        r.project(sc, f)
        ev[1].record()
        r.bin_sort()
        ev[2].record()
        r.render(out, fov=True)
        ev[3].record()
        torch.cuda.synchronize()
        for q, nm in enumerate(("project", "bin_sort", "render")):
            st[nm].append(ev[q].elapsed_time(ev[q + 1]))
    stages = {k: round(float(np.median(v)), 3) for k, v in st.items()}
    # one more staged frame in an NVTX range (what kernel profiles of this
    # workload select)
    torch.cuda.nvtx.range_push("batched_frame")
    frame()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        frame()   # warm the side stream
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=s):
            frame()
    torch.cuda.current_stream().wait_stream(s)
    code, c2 = r.counters()
    ms = _ms(torch, graph.replay, steps, 1, flush)
    code, c3 = r.counters()
    peaks, src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    bs_bytes = bin_sort_bytes(r.n * r.V, int(c["n_visible"]), int(c["n_pairs"]), r.T_tiles,
                              pair_passes(r.T_tiles, opt["radix_bits"]), True, True,
                              depth_passes(r, gs))
    bs_gbs = bs_bytes / (stages["bin_sort"] * 1e-3) / 1e9
    res = {"workload": wl.name, "views": len(wl.cams), "pixels": r.P,
           "ms_per_batch": round(ms, 3), "views_per_s": round(len(wl.cams) * 1000 / ms, 2),
           "gpix_per_s": round(r.P / ms / 1e6, 3), "pairs": int(c["n_pairs"]),
           "visible": int(c["n_visible"]), "status": int(code),
           "kernel_launches_in_graph": r.launches_per_frame(fov=True),
           "stages_ms": stages,
           "roofline_bin_sort": {"bound": "hbm", "achieved": round(bs_gbs, 1), "peak": hbm,
                                 "unit": "GB/s", "frac": round(bs_gbs / hbm, 4),
                                 "bytes_per_batch": int(bs_bytes),
                                 "peak_source": f"{src} hbm_gbs (copy); of measured"},
           "autotuned": opt, "autotune_trials": tune["trials"]}
    del r, graph, out
    torch.cuda.empty_cache()
    if not separate:
        return res
    # the same 64 views as separate single-view plans (one plan per view size
    # and mode, its cameras swapped per view): every view projects all points,
    # bins and sorts its own pairs, renders its own tiles
    sides = wl.cams[:, 16].astype(int)
    vf = wl.fov.view_fov
    plans = {}
    per_out = {}
    for key in sorted(set(zip(sides.tolist(), vf.tolist()))):
        idx = [v for v in range(len(wl.cams)) if (sides[v], vf[v]) == key]
        fv = synth.Foveation(wl.fov.n_levels, wl.fov.bound_m, wl.fov.ring_tan, wl.fov.band_px,
                             wl.fov.gaze[idx[:1]], np.ones(1, np.uint8))
        rv = gs.Renderer(wl.scene.n, 3, wl.cams[idx[0]:idx[0] + 1], foveated=bool(key[1]),
                         tight=True, tile=opt["tile"], radix_bits=opt["radix_bits"],
                         chunk=opt["chunk"])
        fd = gs.fov_to_device(fv) if key[1] else None
        kmax = 0
        for v in idx:
            rv.set_cameras(wl.cams[v:v + 1])
            if fd is not None:
                fd["gaze"].copy_(torch.from_numpy(wl.fov.gaze[v:v + 1]).cuda())
            kmax = max(kmax, int(rv.fit(sc, fd, headroom=1.05)["n_pairs"]))
        plans[key] = (rv, fd, idx)
        per_out[key] = rv.alloc_outputs(fov=bool(key[1]))
    gaze_dev = {v: torch.from_numpy(wl.fov.gaze[v:v + 1]).cuda() for v in range(len(wl.cams))}
    cams_dev = {v: gs.cams_device(wl.cams[v:v + 1]) for v in range(len(wl.cams))}

    def per_view():
        for key, (rv, fd, idx) in plans.items():
            for v in idx:
                rv.cams_d.copy_(cams_dev[v])
                if fd is not None:
                    fd["gaze"].copy_(gaze_dev[v])
                rv.project(sc, fd)
                rv.bin_sort()
                rv.render(per_out[key], fov=fd is not None)

    ms_pv = _ms(torch, per_view, max(2, steps // 2), 1, flush)
    res.update({"ms_per_batch_separate_plans": round(ms_pv, 3),
                "batched_speedup": round(ms_pv / ms, 3)})
    del plans, per_out, sc
    torch.cuda.empty_cache()
    return res


# --------------------------------------------------------------------------
# CPU arm: the FP64 oracle on a bounded sample
# --------------------------------------------------------------------------
def cpu_oracle_fps(budget_s=20.0, all_cores=True):
    """Frames/s of the oracle on the 1080p/1M workload: binning of the whole
    frame plus compositing of a random sample of tiles, scaled to the frame.
    ``all_cores``: the oracle's -fopenmp build (independent items and pixels
    split over the host's cores, same arithmetic); else single-threaded."""
    import numpy as np

    import oracle
    from paper_2407_00435_gb300 import synth
    oracle.build()
    used = oracle.use_all_cores(all_cores)
    try:
        wl = synth.workload(1)
        t0 = time.perf_counter()
        b = oracle.bin_pairs(wl.scene, wl.cams, 16, tight=True)
        t_bin = time.perf_counter() - t0
        vp = oracle.project_values(wl.scene, wl.cams, b.vis)
        t_proj = time.perf_counter() - t0 - t_bin
        rng = np.random.default_rng(0)
        T = len(b.ranges)
        order = rng.permutation(T)
        done_tiles, t_render = 0, 0.0
        step = 64 if used else 1             # tiles per oracle call
        for k in range(0, T, step):
            pix = []
            for t in order[k:k + step]:
                ty, tx = divmod(int(t), 120)
                pix += [y * 1920 + x for y in range(ty * 16, min(1080, ty * 16 + 16))
                        for x in range(tx * 16, tx * 16 + 16)]
            s = time.perf_counter()
            oracle.render(wl.scene, wl.cams, 16, b, pix=np.array(pix, np.int64), vp=vp)
            t_render += time.perf_counter() - s
            done_tiles += len(order[k:k + step])
            if t_bin + t_proj + t_render > budget_s:
                break
        frame_s = t_bin + t_proj + t_render * T / done_tiles
        cores = oracle.threads()
    finally:
        oracle.use_all_cores(False)
    return {"value": round(1.0 / frame_s, 5), "unit": "frames/s", "cores": cores, "kind": "oracle",
            "build": "all cores (-fopenmp over items and pixels)" if used else "single-threaded",
            "sample": f"full-frame binning + FP64 projection, {done_tiles}/{T} random tiles "
                      f"composited and scaled to the frame ({t_bin + t_proj + t_render:.1f} s)",
            **host_info()}


def cpu_baseline():
    """The all-core oracle, with the single-threaded one beside it."""
    allc = cpu_oracle_fps(12.0, all_cores=True)
    one = cpu_oracle_fps(12.0, all_cores=False)
    allc["single_core"] = {k: one[k] for k in ("value", "cores", "sample")}
    return allc


def reference_arm(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per = max(4.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_oracle_fps(per)
    vals = [cpu_oracle_fps(per) for _ in range(args.steps)]
    v = statistics.mean(x["value"] for x in vals)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": "frames/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1000.0 / v, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**HEADLINE_CONFIG, "parallelism": f"replicas x{world}"},
            "cpu_baseline": {**vals[-1], "value": round(v, 5)},
            "e2e": {"value": round(v, 5), "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    res, rank, world = gpu_arm(args)
    if rank == 0:
        if world == 1 and not args.no_cpu:
            res["cpu_baseline"] = cpu_baseline()
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
