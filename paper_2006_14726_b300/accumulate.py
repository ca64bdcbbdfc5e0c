"""Accumulation over server frames: one splat set, one LBVH and one trace for the window of the F
newest server frames (the paper names accumulating frames as future work, §6, without a rule).

Reading (spec S3a): the frame of age g (0 = newest) contributes its splats with colour weight
decay^g and ids offset by g * Ws * Hs, appended newest first, so that newer frames win ties of
equal hit distance; with one frame the set is exactly the plain unprojection.  Every step runs in
the library's kernels: wrs_unproject for the newest frame, wrs_unproject_append for each older one,
wrs_build_lbvh over the union and wrs_trace per client view.
"""
from __future__ import annotations

from collections import deque
from typing import Optional

import torch

from . import (LBVH, LBVH_FULL, RADIUS_FOOTPRINT, SplatBuffers, TraceParams, _cam, _scratch, build_lbvh,
               lbvh_scratch_bytes, new_status, trace, unproject, unproject_append,
               unproject_scratch_bytes, window_weight)


def window_weights(frames: int, decay: float = 1.0):
    """Colour weight of each frame of the window, newest first (wrs_window_weight: decay^g by
    repeated binary32 multiplication, spec S3a)."""
    return [window_weight(decay, g) for g in range(frames)]


class FrameWindow:
    """The splats of the ``frames`` newest server frames (all of one size) in one LBVH.

    ``push`` keeps references to the given device tensors (the caller does not overwrite them
    while they are in the window) and rebuilds the set; ``trace`` renders a client view of it.
    ``layout``: the LBVH's (LBVH_WIDE when every trace walks the 4-wide nodes)."""

    def __init__(self, frames: int, width: int, height: int, decay: float = 1.0,
                 leaf_size: int = 1, radius_mode: int = RADIUS_FOOTPRINT, voxel_diag: float = 0.0,
                 device=None, layout: int = LBVH_FULL):
        if frames < 1:
            raise ValueError("a window holds at least one frame")
        if not (0.0 < decay <= 1.0):
            raise ValueError("decay must lie in (0, 1]")
        device = device or torch.device("cuda")
        self.frames, self.width, self.height = int(frames), int(width), int(height)
        self.npix = self.width * self.height
        if self.frames * self.npix > 2**31:
            raise ValueError("window of more than 2^31 pixels")
        self.weights = window_weights(self.frames, decay)
        self.radius_mode, self.voxel_diag = int(radius_mode), float(voxel_diag)
        self.capacity = self.frames * self.npix
        self.splats = SplatBuffers(self.capacity, device=device)
        self.bvh = LBVH(self.capacity, leaf_size, device=device, layout=layout)
        self.sorted = SplatBuffers(self.capacity, device=device, sorted=True)
        self._uscratch = _scratch(unproject_scratch_bytes(self.width, self.height), device)
        self._bscratch = _scratch(lbvh_scratch_bytes(self.capacity, leaf_size), device)
        self.status = new_status(device)
        self._window = deque(maxlen=self.frames)  # newest first

    def __len__(self) -> int:
        return len(self._window)

    def push(self, rgba: torch.Tensor, depth: torch.Tensor, cam, stream=None):
        """Add the newest server frame (dropping the oldest once full) and rebuild."""
        c = _cam(cam)
        if (c.width, c.height) != (self.width, self.height):
            raise ValueError(f"frame of {c.width}x{c.height}, window of {self.width}x{self.height}")
        self._window.appendleft((rgba, depth, cam))
        self.rebuild(stream)

    def rebuild(self, stream=None):
        """Unproject every frame of the window into the one set (newest first) and build the LBVH."""
        for g, (rgba, depth, cam) in enumerate(self._window):
            if g == 0:
                unproject(rgba, depth, cam, self.radius_mode, self.voxel_diag, out=self.splats,
                          scratch=self._uscratch, stream=stream)
            else:
                unproject_append(rgba, depth, cam, self.splats, self.weights[g], g * self.npix,
                                 self.radius_mode, self.voxel_diag, status=self.status,
                                 scratch=self._uscratch, stream=stream)
        build_lbvh(self.splats, self.bvh.leaf_size, bvh=self.bvh, sorted=self.sorted,
                   scratch=self._bscratch, stream=stream)

    def trace(self, cam, params: TraceParams = TraceParams(), out: Optional[torch.Tensor] = None,
              stream=None) -> torch.Tensor:
        return trace(self.bvh, self.sorted, cam, params, out=out, status=self.status, stream=stream)
