"""Frames whose inputs live in pinned host memory, pipelined over three CUDA
streams: the upload of frame i+1's scene (copy stream) overlaps the
projection, binning and render of frame i (compute stream), and the image
read-back of frame i (read-back stream) overlaps frame i+1's compute.

Scene buffers and output images are rotated over ``depth`` slots; one
workspace serialises the compute stream.  The scene buffer of a slot is
refilled as soon as the projection that read it has finished (the later
stages read only the workspace), and its image once its read-back is done.
Every kernel is the library's; this module only orders copies and calls.
"""
from __future__ import annotations

import torch

from .gs import Renderer

SCENE_KEYS = ("means", "scales", "quats", "opac", "sh")


class HostFramePipeline:
    """``renderer`` must already be fitted (its pair capacity holds the
    frames); ``fov`` is the device foveation dict of gs.fov_to_device or
    None."""

    def __init__(self, renderer: Renderer, fov: dict | None = None, bg=(0.0, 0.0, 0.0),
                 depth: int = 2):
        if depth < 1:
            raise ValueError("depth must be >= 1")
        self.r = renderer
        self.fov = fov
        self.bg = bg
        self.depth = depth
        self.comp = torch.cuda.Stream()
        self.copy = torch.cuda.Stream()
        self.read = torch.cuda.Stream()
        self.dev = [None] * depth
        self.outs = [renderer.alloc_outputs(fov=fov is not None) for _ in range(depth)]
        self._proj = [None] * depth      # projection of the slot's last frame done
        self._read = [None] * depth      # read-back of the slot's last image done

    def _buffers(self, slot, host_scene):
        if self.dev[slot] is None:
            self.dev[slot] = {k: torch.empty(host_scene[k].shape, dtype=host_scene[k].dtype,
                                             device="cuda") for k in SCENE_KEYS}
        return self.dev[slot]

    def run(self, frames, start_event=None, end_event=None):
        """``frames``: iterable of (host scene dict of pinned tensors, pinned
        host rgb tensor (P, 3)).  Enqueues every frame; ``start_event`` is
        recorded on the copy stream before the first upload and
        ``end_event`` after the last read-back (both optional).  Returns
        without synchronising."""
        cur = torch.cuda.current_stream()
        for s in (self.comp, self.copy, self.read):
            s.wait_stream(cur)
        if start_event is not None:
            start_event.record(self.copy)
            self.comp.wait_event(start_event)
            self.read.wait_event(start_event)
        fov = self.fov is not None
        for i, (hs, hrgb) in enumerate(frames):
            slot = i % self.depth
            dev = self._buffers(slot, hs)
            with torch.cuda.stream(self.copy):
                if self._proj[slot] is not None:
                    self.copy.wait_event(self._proj[slot])
                for k in SCENE_KEYS:
                    dev[k].copy_(hs[k], non_blocking=True)
                up = torch.cuda.Event()
                up.record(self.copy)
            self.comp.wait_event(up)
            if self._read[slot] is not None:
                self.comp.wait_event(self._read[slot])
            out = self.outs[slot]
            self.r.project(dev, self.fov, stream=self.comp)
            ev = torch.cuda.Event()
            ev.record(self.comp)
            self._proj[slot] = ev
            self.r.bin_sort(stream=self.comp)
            self.r.render(out, bg=self.bg, fov=fov, stream=self.comp)
            done = torch.cuda.Event()
            done.record(self.comp)
            with torch.cuda.stream(self.read):
                self.read.wait_event(done)
                hrgb.copy_(out["rgb"], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(self.read)
                self._read[slot] = ev
        if end_event is not None:
            self.read.wait_stream(self.comp)
            self.read.wait_stream(self.copy)
            end_event.record(self.read)
        for s in (self.comp, self.copy, self.read):
            cur.wait_stream(s)
