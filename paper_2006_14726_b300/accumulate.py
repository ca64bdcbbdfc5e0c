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


def _torch_stream(stream):
    """A torch stream object for ``stream`` (None: the current stream; a torch stream; or a raw
    cudaStream_t handle)."""
    if stream is None:
        return torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return stream
    return torch.cuda.ExternalStream(int(stream))


def window_weights(frames: int, decay: float = 1.0):
    """Colour weight of each frame of the window, newest first (wrs_window_weight: decay^g by
    repeated binary32 multiplication, spec S3a)."""
    return [window_weight(decay, g) for g in range(frames)]


class FrameWindow:
    """The splats of the ``frames`` newest server frames (all of one size) in one LBVH.

    ``push`` keeps references to the given device tensors (the caller does not overwrite them
    while they are in the window) and rebuilds the set; ``trace`` renders a client view of it.
    ``layout``: the LBVH's (LBVH_WIDE when every trace walks the 4-wide nodes).

    ``slots`` = 2 keeps two copies of the set and its LBVH: a push rebuilds the copy that the
    previous frame's views are not reading, so a push on one stream overlaps the traces still
    running on another (each trace waits for the build of its copy; each rebuild waits for the
    traces of the copy it overwrites and for that copy's last build, whichever streams they ran
    on).  Results do not depend on it."""

    def __init__(self, frames: int, width: int, height: int, decay: float = 1.0,
                 leaf_size: int = 1, radius_mode: int = RADIUS_FOOTPRINT, voxel_diag: float = 0.0,
                 device=None, layout: int = LBVH_FULL, slots: int = 1):
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
        if slots not in (1, 2):
            raise ValueError("slots must be 1 or 2")
        self._slots = []
        for _ in range(slots):
            freed = torch.cuda.Event()
            freed.record()  # nothing reads a fresh copy
            self._slots.append({
                "splats": SplatBuffers(self.capacity, device=device),
                "bvh": LBVH(self.capacity, leaf_size, device=device, layout=layout),
                "sorted": SplatBuffers(self.capacity, device=device, sorted=True),
                "uscratch": _scratch(unproject_scratch_bytes(self.width, self.height), device),
                "bscratch": _scratch(lbvh_scratch_bytes(self.capacity, leaf_size), device),
                "built": torch.cuda.Event(), "freed": freed})
        self._cur = 0
        self.status = new_status(device)
        self._window = deque(maxlen=self.frames)  # newest first

    @property
    def splats(self) -> SplatBuffers:
        """The current splat set (of the last rebuild)."""
        return self._slots[self._cur]["splats"]

    @property
    def bvh(self) -> LBVH:
        return self._slots[self._cur]["bvh"]

    @property
    def sorted(self) -> SplatBuffers:
        return self._slots[self._cur]["sorted"]

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
        """Unproject every frame of the window into the one set (newest first) and build the LBVH
        (into the other copy when there are two)."""
        k = (self._cur + 1) % len(self._slots)
        sl = self._slots[k]
        st = _torch_stream(stream)
        st.wait_event(sl["freed"])  # the traces that read this copy have finished
        st.wait_event(sl["built"])  # and its last build, which may have run on another stream
        for g, (rgba, depth, cam) in enumerate(self._window):
            if g == 0:
                unproject(rgba, depth, cam, self.radius_mode, self.voxel_diag, out=sl["splats"],
                          scratch=sl["uscratch"], stream=st)
            else:
                unproject_append(rgba, depth, cam, sl["splats"], self.weights[g], g * self.npix,
                                 self.radius_mode, self.voxel_diag, status=self.status,
                                 scratch=sl["uscratch"], stream=st)
        build_lbvh(sl["splats"], sl["bvh"].leaf_size, bvh=sl["bvh"], sorted=sl["sorted"],
                   scratch=sl["bscratch"], stream=st)
        sl["built"].record(st)
        self._cur = k

    def trace(self, cam, params: TraceParams = TraceParams(), out: Optional[torch.Tensor] = None,
              stream=None) -> torch.Tensor:
        sl = self._slots[self._cur]
        st = _torch_stream(stream)
        st.wait_event(sl["built"])
        img = trace(sl["bvh"], sl["sorted"], cam, params, out=out, status=self.status, stream=st)
        sl["freed"].record(st)
        return img
