"""The client of the remote renderer as a stream pipeline: server frames come in from host memory,
warped client views go back to host memory, and the copies overlap the GPU work.

The paper's client receives each server frame (colour + depth + camera) over the network, rebuilds
its sphere splats and LBVH, and keeps rendering novel views from the newest frame while the next
one arrives (§4, §4.2).  Here the network is replaced by pinned host buffers; the pipeline keeps
three CUDA streams:

* ``h2d``: copies of incoming server frames into one of two device scene slots;
* ``compute``: unprojection + LBVH build of a slot (the build replayed from a CUDA graph captured
  per slot), then the traces of client views;
* ``d2h``: copies of finished views into a ring of pinned host images.

A scene slot is rebuilt only after the traces that read it have finished, and an image slot of the
ring is overwritten only after its previous copy to the host has finished, so every ordering is an
event dependency between streams; the host blocks only in :meth:`WarpingClient.result` (and when
the ring wraps onto an image nobody has collected).  Every step runs in the library's kernels.
"""
from __future__ import annotations

from typing import List, Optional

import torch

from . import (LBVH, RADIUS_FOOTPRINT, SplatBuffers, TraceParams, build_lbvh, lbvh_scratch_bytes,
               make_camera, new_status, trace, tree_layout, unproject, unproject_scratch_bytes)


class _Scene:
    def __init__(self, sw: int, sh: int, leaf: int, device, layout: int):
        npix = sw * sh
        self.rgba = torch.empty(sh, sw, 4, dtype=torch.float32, device=device)
        self.depth = torch.empty(sh, sw, dtype=torch.float32, device=device)
        self.splats = SplatBuffers(npix, device=device)
        self.bvh = LBVH(npix, leaf, device=device, layout=layout)
        self.sorted = SplatBuffers(npix, device=device, sorted=True)
        self.uscratch = torch.empty(max(unproject_scratch_bytes(sw, sh), 256), dtype=torch.uint8,
                                    device=device)
        self.bscratch = torch.empty(max(lbvh_scratch_bytes(npix, leaf), 256), dtype=torch.uint8,
                                    device=device)
        self.copied = torch.cuda.Event()
        self.built = torch.cuda.Event()     # the slot's splats and LBVH are complete
        self.released = torch.cuda.Event()  # the last trace that read this slot has finished
        self.released.record()              # (nothing reads a fresh slot)
        # the slot's LBVH build reads and writes only the slot's own buffers (the splat count
        # stays on the device), so one CUDA graph of its launches serves every frame
        self.build = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(device=device)
        side.wait_stream(torch.cuda.current_stream(device))
        with torch.cuda.stream(side):
            with torch.cuda.graph(self.build, stream=side):
                build_lbvh(self.splats, leaf, bvh=self.bvh, sorted=self.sorted,
                           scratch=self.bscratch, stream=side)
        torch.cuda.current_stream(device).wait_stream(side)


class WarpingClient:
    """Overlapped host → device → host pipeline of the warping client.

    ``submit(rgba, depth, cam)`` takes a server frame in pinned host memory (premultiplied RGBA
    [Hs, Ws, 4] float32, depth [Hs, Ws] float32, the server camera) and queues its copy, splats and
    LBVH; ``render(cam)`` queues a client view of the newest submitted frame and its copy back,
    returning a ticket; ``result(ticket)`` waits for that copy and returns the pinned host image
    (valid until the ring of ``ring`` images wraps onto it).  Four streams: host → device copies,
    the splats and LBVH of a new frame (a stream of higher priority, so that they overlap the
    views still being traced from the previous frame), the traces, and device → host copies."""

    def __init__(self, server_w: int, server_h: int, client_w: int, client_h: int,
                 params: TraceParams = TraceParams(width=4, k_chunk=1), leaf_size: int = 1,
                 ring: int = 8, radius_mode: int = RADIUS_FOOTPRINT, voxel_diag: float = 0.0,
                 device=None):
        device = device or torch.device("cuda")
        self.params = params
        self.leaf = int(leaf_size)
        self.radius_mode, self.voxel_diag = int(radius_mode), float(voxel_diag)
        self.sw, self.sh, self.cw, self.ch = int(server_w), int(server_h), int(client_w), int(client_h)
        self.compute = torch.cuda.Stream(device=device)
        self.build = torch.cuda.Stream(device=device, priority=-1)  # the higher priority
        self.h2d = torch.cuda.Stream(device=device)
        self.d2h = torch.cuda.Stream(device=device)
        # a client that walks the 4-wide nodes builds trees without the binary records
        self.scenes = [_Scene(self.sw, self.sh, self.leaf, device, tree_layout(params))
                       for _ in range(2)]
        self.current: Optional[int] = None
        self.status = new_status(device)
        self.dev_out = [torch.empty(self.ch, self.cw, 4, dtype=torch.float32, device=device)
                        for _ in range(ring)]
        self.host_out = [torch.empty(self.ch, self.cw, 4, dtype=torch.float32).pin_memory()
                         for _ in range(ring)]
        self.traced = [torch.cuda.Event() for _ in range(ring)]
        self.copied = [torch.cuda.Event() for _ in range(ring)]
        self.pending: List[bool] = [False] * ring
        self.ticket = 0

    # ---- server frames ------------------------------------------------------------------------
    def submit(self, h_rgba: torch.Tensor, h_depth: torch.Tensor, cam):
        """Queue a new server frame; later renders use it."""
        slot = 0 if self.current is None else 1 - self.current
        sc = self.scenes[slot]
        self.h2d.wait_event(sc.released)  # traces of the frame this slot held have finished
        with torch.cuda.stream(self.h2d):
            sc.rgba.copy_(h_rgba, non_blocking=True)
            sc.depth.copy_(h_depth, non_blocking=True)
        sc.copied.record(self.h2d)
        self.build.wait_event(sc.copied)
        unproject(sc.rgba, sc.depth, cam, self.radius_mode, self.voxel_diag, out=sc.splats,
                  scratch=sc.uscratch, stream=self.build)
        with torch.cuda.stream(self.build):
            sc.build.replay()
        sc.built.record(self.build)
        self.current = slot

    # ---- client views -------------------------------------------------------------------------
    def render(self, cam) -> int:
        """Queue the view of ``cam`` from the newest frame and its copy to the host; returns a
        ticket for :meth:`result`."""
        if self.current is None:
            raise RuntimeError("render before the first server frame")
        k = self.ticket % len(self.dev_out)
        if self.pending[k]:               # the ring wrapped onto an image nobody collected
            self.copied[k].synchronize()
        self.compute.wait_event(self.copied[k])  # its previous copy out has finished
        sc = self.scenes[self.current]
        self.compute.wait_event(sc.built)
        trace(sc.bvh, sc.sorted, make_camera(cam), self.params, out=self.dev_out[k],
              status=self.status, stream=self.compute)
        self.traced[k].record(self.compute)
        sc.released.record(self.compute)
        self.d2h.wait_event(self.traced[k])
        with torch.cuda.stream(self.d2h):
            self.host_out[k].copy_(self.dev_out[k], non_blocking=True)
        self.copied[k].record(self.d2h)
        self.pending[k] = True
        t = self.ticket
        self.ticket += 1
        return t

    def result(self, ticket: int) -> torch.Tensor:
        """Wait for the view of ``ticket`` to reach the host; returns its pinned host image."""
        if ticket < self.ticket - len(self.dev_out) or ticket >= self.ticket:
            raise ValueError("ticket is no longer (or not yet) in the ring")
        k = ticket % len(self.dev_out)
        self.copied[k].synchronize()
        self.pending[k] = False
        return self.host_out[k]

    def synchronize(self):
        """Wait for all queued work of the three streams."""
        for s in (self.h2d, self.build, self.compute, self.d2h):
            s.synchronize()
        self.pending = [False] * len(self.pending)
