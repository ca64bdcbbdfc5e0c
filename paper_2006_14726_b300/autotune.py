"""Autotuner for the performance knobs of the trace: LBVH leaf size, k-buffer depth, block size,
node width and schedule (one thread per pixel, persistent blocks with lane refill, or one
warp-shared traversal per 8x4 tile).

The knobs never change results (the hit set and order are fixed by the binary32 sphere test; the
compositing visits hits in that order), so the tuner only measures time: it builds one LBVH per
leaf size, times wrs_trace (or wrs_trace_batched) over the given cameras with CUDA events, and
keeps the fastest combination.  Choices are cached per GPU model and workload signature in a
small JSON file (``$WRS_AUTOTUNE_CACHE``, default ``~/.cache/wrs/autotune.json``).
"""
from __future__ import annotations

import json
import os
from typing import Callable, Dict, Iterable, Optional, Sequence

import torch

from . import (LBVH_WIDE, SCHEDULE_PACKET, SCHEDULE_PER_PIXEL, SCHEDULE_PER_SESSION,
               SCHEDULE_PERSISTENT, Batch, SplatBuffers, TraceParams, build_lbvh, trace,
               trace_batched, version)

LEAVES = (1, 2, 4)
KS = (1, 2, 4, 8)
BLOCKS = (64, 128, 256)
WIDTHS = (2, 4)


def _cache_path() -> str:
    return os.environ.get("WRS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "wrs", "autotune.json"))


def _load_cache() -> dict:
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, val: dict):
    try:
        c = _load_cache()
        c[key] = val
        os.makedirs(os.path.dirname(_cache_path()), exist_ok=True)
        with open(_cache_path(), "w") as f:
            json.dump(c, f, indent=1)
    except OSError:
        pass


def _time_ms(fn: Callable[[], None], reps: int, warm: int = 2) -> float:
    for _ in range(warm):
        fn()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def signature(kind: str, n_splats: int, width: int, height: int, base: TraceParams) -> str:
    gpu = torch.cuda.get_device_name()
    nb = 1 << max(0, int(n_splats).bit_length() - 1)  # power-of-two bucket of the splat count
    # the library version is part of the key: a choice measured on other kernels is not reused
    return (f"{version()}|{gpu}|{kind}|n~{nb}|{width}x{height}|H{base.max_hits}"
            f"|b{base.edge_softness:g}")


def tune_trace(splats: SplatBuffers, cams: Sequence, base: TraceParams = TraceParams(),
               leaves: Iterable[int] = LEAVES, ks: Iterable[int] = KS,
               blocks: Iterable[int] = BLOCKS, widths: Iterable[int] = WIDTHS, reps: int = 3,
               use_cache: bool = True, build_weight: float = 0.0) -> Dict:
    """Pick (leaf_size, k_chunk, block, schedule, width) minimising the mean wrs_trace time over
    ``cams`` plus ``build_weight`` times the LBVH build time of the leaf size (the share of a
    build per traced view, e.g. 1/4 when a server frame serves four client views).  A launch
    that walks the 4-wide nodes is charged the build of the 4-wide-only layout (LBVH_WIDE), the
    binary traversal the full one."""
    c0 = cams[0]
    key = signature("trace", splats.count(), c0.width, c0.height, base) + f"|w{build_weight:g}"
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return hit
    best = None
    table = []
    for leaf in leaves:
        bvh, srt = build_lbvh(splats, leaf)
        build_ms = _time_ms(lambda: build_lbvh(splats, leaf, bvh=bvh, sorted=srt), reps)
        wb, ws = build_lbvh(splats, leaf, layout=LBVH_WIDE)
        build_wide_ms = _time_ms(lambda: build_lbvh(splats, leaf, bvh=wb, sorted=ws), reps)
        del wb, ws
        outs = [torch.empty(c.height, c.width, 4, device=splats.pos_r.device) for c in cams]
        shapes = [(b, SCHEDULE_PER_PIXEL) for b in blocks] + [(128, SCHEDULE_PERSISTENT),
                                                              (128, SCHEDULE_PACKET)]
        for k in ks:
            for block, sched in shapes:
                # the packet schedule always walks the 4-wide nodes
                for width in (widths if sched != SCHEDULE_PACKET else (4,)):
                    p = TraceParams(base.max_hits, base.t_stop, base.edge_softness, k, block, sched,
                                    width)

                    def run():
                        for c, o in zip(cams, outs):
                            trace(bvh, srt, c, p, out=o)
                    ms = _time_ms(run, reps) / len(cams)
                    bms = build_wide_ms if (width == 4 or sched == SCHEDULE_PACKET) else build_ms
                    score = ms + build_weight * bms
                    table.append((leaf, k, block, sched, width, ms, bms))
                    if best is None or score < best["score"]:
                        best = {"leaf": leaf, "k_chunk": k, "block": block, "schedule": sched,
                                "width": width, "ms": ms, "build_ms": bms, "score": score}
    best["table"] = table
    _store(key, best)
    return best


def tune_batched(batch: Batch, base: TraceParams = TraceParams(), ks: Iterable[int] = KS,
                 widths: Iterable[int] = WIDTHS, reps: int = 3) -> Dict:
    """Pick (k_chunk, width, schedule) for one multi-session launch (leaf sizes are fixed by the
    sessions' LBVHs; blocks of 128 threads: one warp per tile, one warp-shared traversal per
    tile, each session's own schedule of the two (``batch.schedules``), or one resident wave
    with lane refill)."""
    best = None
    for sched in (SCHEDULE_PER_PIXEL, SCHEDULE_PERSISTENT, SCHEDULE_PACKET, SCHEDULE_PER_SESSION):
        for k in ks:
            # the packet schedule always walks the 4-wide nodes
            for width in (widths if sched != SCHEDULE_PACKET else (4,)):
                p = TraceParams(base.max_hits, base.t_stop, base.edge_softness, k, 128, sched, width)
                ms = _time_ms(lambda: trace_batched(batch, p), reps)
                if best is None or ms < best["ms"]:
                    best = {"k_chunk": k, "block": 128, "width": width, "schedule": sched, "ms": ms}
    return best
