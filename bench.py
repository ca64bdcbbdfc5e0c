#!/usr/bin/env python
"""Benchmark of the sphere-splat warping hot path on B300.

One step = one new server depth image of the large workload followed by its frames:
unproject (Eq. 1, footprint radius, compaction) + LBVH rebuild + 4 client frames traced and
composited (1920x1080 server image of a 512^3 u8 Fourier volume, about 2.07 M splats, 1920x1080
client, poses within 20 degrees, a new depth image every 4 frames).  value = client primary rays
per second over the whole job (all ranks), Mrays/s, of K steps run as a client runs them: the next
frame's unproject and LBVH build (two buffer slots, a build stream of higher priority) overlap
this frame's 4 traces.  The same K steps one after another on one stream are reported as
`sequential`, with the stage split.

Also reported on the same line: LBVH build and unproject ms, trace-only Mrays/s, the roofline of
the trace kernel, the batched workload (64 sessions, one launch replayed from a CUDA graph vs 64
sequential calls), accumulation over a window of the 4 newest server frames (one LBVH and one
trace over their union), forward and forward+backward throughput of the differentiable renderer,
an end-to-end number through host buffers, and the CPU oracle timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl wrs|reference] [--no-extras]

Multi-GPU (torchrun): every rank runs its own replica of the workload on its own poses (weak
scaling, no collective on the data path); time = max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1080p/2M-splat Mrays/s & LBVH ms; batched and fwd+bwd vs plain, % roofline"
UNIT = "Mrays/s"
FRAMES_PER_IMAGE = 4
SCHEDULE_NAMES = ["one thread per pixel", "persistent, lane refill", "packet, one traversal per warp"]
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="wrs", choices=["wrs", "reference"])
    ap.add_argument("--no-extras", action="store_true",
                    help="skip batched / fwd+bwd / e2e / cpu baseline (main line only)")
    ap.add_argument("--sizes", action="store_true",
                    help="instead of the benchmark line, print one JSON line with the size "
                         "scaling of unproject + LBVH (server 512^2 .. 4096^2) and of the trace "
                         "(client 256^2 .. 4096^2 on the 1080p server frame), large workload "
                         "volume, warm L2, 10 repetitions each")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the launch the tuner picks on B300 (leaf 1, K 1, 128 threads per "
                         "pixel, 4-wide nodes) instead of tuning; for profiler runs, where tuning "
                         "times are distorted")
    cs = ap.add_argument_group("profiling cases (--case): one workload once, few launches")
    cs.add_argument("--case", choices=["tiny", "mid", "large", "diff", "batched"],
                    help="instead of the benchmark line, run one workload once with few launches "
                         "(for ncu) and print its CUDA event times")
    cs.add_argument("--groups", default="",
                    help="large/mid: comma-separated depth-image groups; each group ray-casts its "
                         "own server image and traces --frames of its poses (default: the "
                         "server camera and the first --frames poses)")
    cs.add_argument("--sessions", type=int, default=16)
    cs.add_argument("--frames", type=int, default=3)
    cs.add_argument("--leaf", type=int, default=1)
    cs.add_argument("--k", type=int, default=1)
    cs.add_argument("--block", type=int, default=128)
    cs.add_argument("--max-hits", type=int, default=0)
    cs.add_argument("--schedule", type=int, default=0, help="0 per pixel, 1 persistent, 2 packet")
    cs.add_argument("--width", type=int, default=4, help="2 binary nodes, 4 four-wide nodes")
    cs.add_argument("--layout", choices=["auto", "full", "wide"], default="auto",
                    help="large/mid/tiny: LBVH layout (auto: the 4-wide-only layout when the "
                         "traces walk the 4-wide nodes, as in the benchmark)")
    cs.add_argument("--retraverse", action="store_true",
                    help="diff: the adjoint traces every ray again (no recorded hit lists)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(W, n_splats=None, extra=None):
    cfg = {"workload": W.name, "volume": f"{W.vol_n}^3 u8, {W.vol_param} Fourier modes",
           "server": [W.server_w, W.server_h], "client": [W.client_w, W.client_h],
           "frames_per_depth_image": FRAMES_PER_IMAGE, "poses": f"{W.n_poses} within {W.cap_deg:g} deg",
           "radius": "pixel footprint", "compositing": "all hits front to back, T_stop 1e-5"}
    if n_splats is not None:
        cfg["splats"] = int(n_splats)
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------------------------------------------
# clocks
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # the samples go to $WRS_CLOCKS_DIR (default: the system's temporary directory)
        folder = os.environ.get("WRS_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(folder, f"wrs_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------------------------
# roofline helpers
# ------------------------------------------------------------------------------------------------
def trace_bytes_per_ray(c, rays, width=2):
    """Algorithmic bytes per ray of the trace kernel: per node visited 64 (binary: two child boxes
    and references) or 112 (4-wide: four boxes and references), 16 per sphere tested (centre +
    radius), 4 per hit gathered (its id, for the tie-break), 16 per hit composited (its RGBA), 16
    for the output pixel."""
    node = 112 if width == 4 else 64
    return (node * c["nodes"] + 16 * c["spheres"] + 4 * c["gathered"] + 16 * c["composited"]) / rays + 16


def trace_flops_per_ray(c, rays):
    """22 flops per box test (6 FMA + 10 min/max), 24 per sphere test, 8 per composited hit."""
    return (22 * c["boxes"] + 24 * c["spheres"] + 8 * c["composited"]) / rays


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def launched_block(block, k_chunk, width, schedule):
    """The block size a trace launch runs: the 4-wide per-pixel kernel with K 1, 2, 4 or 8 is
    built for blocks of at most 128 threads, and the library clamps the asked size to it."""
    return min(block, 128) if (width == 4 and k_chunk in (1, 2, 4, 8) and schedule == 0) else block


def lbvh_bytes_per_splat(leaf, full_layout, per_splat_scale=False):
    """Algorithmic DRAM bytes of one LBVH build per splat, kernel by kernel: bounds (read pos_r
    16, + 4 per-splat scale), Morton codes (read 16, write key and index 8), three digit
    histograms (read keys 3 x 4), four scatter passes (read and write key and index, 4 x 16),
    Karras (read keys 4; write node range 16 and parent links 8, + child references 16 in the
    full layout), the visit counters (4), the refit (read order 4, pos_r 16, rgba 16, id 4,
    parent links 8 and node range 16 (+ scale 4); write the sorted splats 40, the 4-wide node
    128, + the binary record's boxes 48 in the full layout).  Per-leaf items scale by 1/leaf."""
    per_splat = 16 + 24 + 12 + 64 + 4 + 16 + 4 + 16 + 4 + 40 + (8 if per_splat_scale else 0)
    per_leaf = 16 + 8 + 4 + 8 + 16 + 128 + (16 + 48 if full_layout else 0)
    return per_splat + per_leaf / leaf


def tree_layout(wrs, width, schedule):
    """The LBVH layout a launch needs: the 4-wide nodes only, unless it walks the binary nodes."""
    return wrs.tree_layout(wrs.TraceParams(schedule=schedule, width=width))


def kernel_digest():
    """Digest of the trace kernel's code (trace.cu and common.cuh with comments, blank lines and
    trailing spaces removed), so that a profile stays attached to the code it measured."""
    import re
    h = hashlib.sha256()
    for p in ("paper_2006_14726_b300/csrc/trace.cu", "paper_2006_14726_b300/csrc/common.cuh"):
        with open(os.path.join(ROOT, p), encoding="utf-8") as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        lines = [ln.rstrip() for ln in src.splitlines()]
        h.update("\n".join(ln for ln in lines if ln).encode())
    return h.hexdigest()[:16]


def profiled(key):
    """A figure of the committed ncu summary of the trace kernel (``- key: value`` lines, means
    per captured launch), if the summary was taken on the current kernel source (it records the
    source digest); else None."""
    path = os.path.join(ROOT, "profiles", "trace_large_1080p_bench_poses.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_digest") != kernel_digest():
        return None
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


def profiled_traffic():
    """DRAM bytes per trace launch (dram__bytes_read.sum + dram__bytes_write.sum) or None."""
    return profiled("dram_bytes_per_launch")


# ------------------------------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ------------------------------------------------------------------------------------------------
def oracle_step_time(rgba_np, depth_np, srv, clis, ray_stride, threads=0):
    """Time one step of the oracle: unproject + its BVH build over all splats + trace of every
    ray_stride-th pixel of each client frame.  Returns (seconds for the full step extrapolated
    from the sampled rays, rays of the full step, detail)."""
    import oracle
    t0 = time.perf_counter()
    sp = oracle.unproject(rgba_np, depth_np, srv)
    t1 = time.perf_counter()
    scene = oracle.Scene(sp)
    bvh = oracle.BVH(scene)
    t2 = time.perf_counter()
    t_trace = 0.0
    rays_full = 0
    for c in clis:
        npix = c.width * c.height
        pix = np.arange(0, npix, ray_stride, dtype=np.int32)
        s = time.perf_counter()
        oracle.trace(scene, c, pixels=pix, bvh=bvh, threads=threads)
        t_trace += (time.perf_counter() - s) * (npix / pix.size)
        rays_full += npix
    total = (t1 - t0) + (t2 - t1) + t_trace
    return total, rays_full, {"unproject_s": t1 - t0, "bvh_s": t2 - t1, "trace_s_extrapolated": t_trace,
                              "splats": sp.n}


def oracle_views(vol_np, tf_np, cams):
    """Reference images of the differentiation workload's fit: the oracle's volume ray caster
    (binary64 compositing, spec S2) at each camera, as float32 tensors [V,H,W,4] on the host.
    Cached in $WRS_CACHE_DIR (default: the system's temporary directory) under a hash of the
    volume, transfer function, cameras and oracle source."""
    import torch
    import oracle
    oracle.build()
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(vol_np).tobytes())
    h.update(np.ascontiguousarray(tf_np, np.float32).tobytes())
    for c in cams:
        h.update(repr((tuple(c.eye), tuple(c.right), tuple(c.up), tuple(c.fwd), c.tan_half_fovy,
                       c.width, c.height)).encode())
    with open(os.path.join(ROOT, "oracle", "oracle.c"), "rb") as f:
        h.update(f.read())
    folder = os.environ.get("WRS_CACHE_DIR") or tempfile.gettempdir()
    path = os.path.join(folder, f"wrs_oracle_views_{h.hexdigest()[:20]}.npy")
    if os.path.exists(path):
        imgs = np.load(path)
    else:
        imgs = np.stack([oracle.raycast(vol_np, tf_np, c)[0].astype(np.float32) for c in cams])
        os.makedirs(folder, exist_ok=True)
        tmp = path + f".tmp{os.getpid()}.npy"
        np.save(tmp, imgs)
        os.replace(tmp, path)
    return list(torch.from_numpy(imgs))


def parity_budget(wrs, torch, synth, params, leaf, pose=5):
    """The tolerance clause on one full 1080p frame in the benchmark's launch: the GPU image
    against the binary64-decision oracle (trace64) on the 1080p stand-in server image (seeded, no
    ray caster, about 2 M splats) at one client pose of the large workload's cap.  Excluded =
    pixels beyond max abs 2e-3; all must be ties (a move of 1e-6 changes their hit list)."""
    import oracle
    rgba, depth = synth.synthetic_server_image(1920, 1080, 52)
    srv = synth.LARGE.server_cam()
    cli = synth.LARGE.client_poses()[pose]
    sp = wrs.unproject(torch.from_numpy(rgba).cuda(), torch.from_numpy(depth).cuda(), srv)
    bvh, srt = wrs.build_lbvh(sp, leaf)
    img = wrs.trace(bvh, srt, cli, params).cpu().numpy().reshape(-1, 4).astype(np.float64)
    ref = oracle.trace64(oracle.Scene(oracle.unproject(rgba, depth, srv)), cli)
    err = np.abs(img - ref["rgba"])
    worst = err.max(1)
    excl = worst > 2e-3
    rest = err[~excl]
    npix = worst.size
    return {"workload": f"1080p stand-in server image (seeded, {sp.count()} splats), client pose "
                        f"{pose} of the large workload's 20 deg cap, the benchmark's launch",
            "oracle": "binary64 decisions (trace64)", "pixels": npix,
            "tie_pixels": int(ref["tie"].sum()), "tie_frac": float(ref["tie"].mean()),
            "excluded_pixels": int(excl.sum()), "excluded_frac": float(excl.sum() / npix),
            "excluded_all_ties": bool(not np.any(excl & ~ref["tie"])),
            "max_abs_rest": float(rest.max()), "mean_abs_rest": float(rest.mean()),
            "tolerance": "max abs 2e-3, mean abs 1e-4 per RGBA channel; exclusions only tie "
                         "pixels, at most 0.1 %"}


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on the host cores, on a bounded sample of
    the large workload per step (server and client downsampled per axis; same volume, cameras and
    depth heuristic; every 4th ray traced), rank 0 only."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import synth
    oracle.build()
    W = synth.LARGE
    down = 4
    vol = W.volume()
    tf = synth.tf_ramp()
    poses = W.client_poses()
    groups = []
    for g in range(2):
        srv = poses[FRAMES_PER_IMAGE * g].with_size(W.server_w // down, W.server_h // down)
        rgba, depth = oracle.raycast(vol, tf, srv)
        clis = [poses[FRAMES_PER_IMAGE * g + f].with_size(W.client_w // down, W.client_h // down)
                for f in range(FRAMES_PER_IMAGE)]
        groups.append((rgba.astype(np.float32), depth, srv, clis))
    threads = oracle.default_threads()
    times = []
    rays = 0
    for s in range(args.warmup + args.steps):
        rgba, depth, srv, clis = groups[s % len(groups)]
        t, r, _ = oracle_step_time(rgba, depth, srv, clis, ray_stride=4, threads=threads)
        if s >= args.warmup:
            times.append(t)
            rays += r
    total = sum(times)
    value = rays / total / 1e6
    sample = (f"server and client {W.server_w // down}x{W.server_h // down} (1/{down} per axis of the "
              f"1920x1080 workload), every 4th ray traced and the trace time scaled to all rays; "
              f"unproject and BVH build over all splats")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(W, extra={"sample": sample, "parallelism": "replicas"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    rank, world, local = dist_env()
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU path)")
    torch.cuda.set_device(local)
    import paper_2006_14726_b300 as wrs
    if args.case:
        run_case(args, wrs, torch)
        return
    if args.sizes:
        if rank == 0:
            print(json.dumps(size_scaling(wrs, torch)), flush=True)
        return
    from paper_2006_14726_b300 import autotune
    from paper_2006_14726_b300.replicas import Replicas
    import synth

    reps = Replicas.from_env("nccl")
    barrier = reps.barrier
    max_over_ranks = reps.max_over_ranks

    W = synth.LARGE
    dev = torch.device("cuda")
    # ---------------- inputs (untimed): volume, poses, server images from the GPU ray caster ---
    vol = torch.from_numpy(W.volume()).to(dev)
    tf = torch.from_numpy(synth.tf_ramp()).to(dev)
    poses = W.client_poses(seed_offset=reps.pose_seed_offset())
    n_groups = len(poses) // FRAMES_PER_IMAGE
    groups = []
    for g in range(n_groups):
        srv = poses[FRAMES_PER_IMAGE * g].with_size(W.server_w, W.server_h)
        rgba, depth = wrs.raycast_volume(vol, tf, srv)
        groups.append((rgba, depth, srv, [wrs.make_camera(poses[FRAMES_PER_IMAGE * g + f])
                                           for f in range(FRAMES_PER_IMAGE)]))
    torch.cuda.synchronize()
    npix_s = W.server_w * W.server_h
    npix_c = W.client_w * W.client_h
    rays_per_step = FRAMES_PER_IMAGE * npix_c

    # ---------------- autotune (untimed; the knobs do not change results) ----------------------
    sp = wrs.unproject(groups[0][0], groups[0][1], groups[0][2])
    if args.no_autotune:
        tuned = {"leaf": 1, "k_chunk": 1, "block": 128, "schedule": 0, "width": 4}
    else:
        # the step builds one LBVH per 4 traced views: tune the whole step, not the trace alone
        tuned = autotune.tune_trace(sp, groups[0][3], use_cache=False,
                                    build_weight=1.0 / FRAMES_PER_IMAGE)
    leaf, kc, block, sched = tuned["leaf"], tuned["k_chunk"], tuned["block"], tuned["schedule"]
    width = tuned["width"]
    params = wrs.TraceParams(max_hits=0, t_stop=1e-5, k_chunk=kc, block=block, schedule=sched,
                             width=width)

    # ---------------- buffers, allocated once -------------------------------------------------
    splats = wrs.SplatBuffers(npix_s)
    layout = tree_layout(wrs, width, sched)
    bvh = wrs.LBVH(npix_s, leaf, layout=layout)
    srt = wrs.SplatBuffers(npix_s, sorted=True)
    up_scratch = torch.empty(wrs.unproject_scratch_bytes(W.server_w, W.server_h), dtype=torch.uint8, device=dev)
    bv_scratch = torch.empty(wrs.lbvh_scratch_bytes(npix_s, leaf), dtype=torch.uint8, device=dev)
    outs = [torch.empty(W.client_h, W.client_w, 4, device=dev) for _ in range(FRAMES_PER_IMAGE)]
    status = wrs.new_status()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    launches_per_step = 3 + 16 + FRAMES_PER_IMAGE  # unproject 3, LBVH 16 kernels, traces

    build_graph = []  # the LBVH build as a CUDA graph, once captured

    def step(g, ev=None):
        rgba, depth, srv, clis = groups[g % n_groups]
        if ev:
            ev[0].record(stream)
        wrs.unproject(rgba, depth, srv, out=splats, scratch=up_scratch, stream=stream)
        if ev:
            ev[1].record(stream)
        if build_graph:
            build_graph[0].replay()
        else:
            wrs.build_lbvh(splats, leaf, bvh=bvh, sorted=srt, scratch=bv_scratch, stream=stream)
        if ev:
            ev[2].record(stream)
        for f in range(FRAMES_PER_IMAGE):
            wrs.trace(bvh, srt, clis[f], params, out=outs[f], status=status, stream=stream)
            if ev:
                ev[3 + f].record(stream)

    # roofline counts over every pose the timed loop visits (untimed)
    cnt_tot = {k: 0 for k in wrs.COUNTER_NAMES}
    rays_counted = 0
    n_splats = []
    for g in range(n_groups):
        step(g)
        n_splats.append(splats.count())
        for c in groups[g][3]:
            cc = wrs.trace_count(bvh, srt, c, params)
            for k in cc:
                cnt_tot[k] += cc[k]
            rays_counted += npix_c
    wrs.check_status(status)

    # The build reads and writes the same buffers every step (the splat count stays on the
    # device), so one CUDA graph replays its 16 launches without launch gaps.
    bg = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        with torch.cuda.graph(bg, stream=side):
            wrs.build_lbvh(splats, leaf, bvh=bvh, sorted=srt, scratch=bv_scratch, stream=side)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    build_graph.append(bg)

    # A second buffer slot for the pipelined loop: the next server frame's unproject and LBVH
    # build (on a build stream of higher priority) run while this frame's client views trace, as
    # a client does when a new frame arrives while it renders the last one.
    slots = [(splats, bvh, srt, up_scratch, bv_scratch, bg)]
    sp2, srt2 = wrs.SplatBuffers(npix_s), wrs.SplatBuffers(npix_s, sorted=True)
    bvh2 = wrs.LBVH(npix_s, leaf, layout=layout)
    up2 = torch.empty_like(up_scratch)
    bv2 = torch.empty_like(bv_scratch)
    wrs.unproject(*groups[0][:3], out=sp2, scratch=up2, stream=stream)
    wrs.build_lbvh(sp2, leaf, bvh=bvh2, sorted=srt2, scratch=bv2, stream=stream)
    bg2 = torch.cuda.CUDAGraph()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        with torch.cuda.graph(bg2, stream=side):
            wrs.build_lbvh(sp2, leaf, bvh=bvh2, sorted=srt2, scratch=bv2, stream=side)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    slots.append((sp2, bvh2, srt2, up2, bv2, bg2))
    bstream = torch.cuda.Stream(priority=-1)  # the higher of the two priorities
    built = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]

    def pipelined(g0, steps):
        """``steps`` whole steps, frame g's unproject + build overlapping frame g-1's traces."""
        for e in freed:
            e.record(stream)
        bstream.wait_stream(stream)
        for i in range(steps + 1):
            if i < steps:
                k = i % 2
                sp_k, _, _, us_k, _, g_k = slots[k]
                rgba, depth, srv, _ = groups[(g0 + i) % n_groups]
                bstream.wait_event(freed[k])  # the traces of the frame this slot held are done
                wrs.unproject(rgba, depth, srv, out=sp_k, scratch=us_k, stream=bstream)
                with torch.cuda.stream(bstream):
                    g_k.replay()
                built[k].record(bstream)
            if i >= 1:
                k = (i - 1) % 2
                _, b_k, s_k, _, _, _ = slots[k]
                stream.wait_event(built[k])
                for f, c in enumerate(groups[(g0 + i - 1) % n_groups][3]):
                    wrs.trace(b_k, s_k, c, params, out=outs[f], status=status, stream=stream)
                freed[k].record(stream)
        stream.wait_stream(bstream)

    for s in range(args.warmup):
        step(s)
    pipelined(0, max(args.warmup, 3))
    torch.cuda.synchronize()

    nev = 3 + FRAMES_PER_IMAGE
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(nev)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed")
    for s in range(args.steps):
        flush.zero_()  # evict L2 before every step (outside the step's events)
        step(s, events[s])
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    # the headline: the same steps pipelined (L2 not flushed: every step reads the next of the
    # 15 server images, 622 MB in rotation, and rebuilds a 0.4 GB tree)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    wall0_p = time.perf_counter()
    torch.cuda.nvtx.range_push("pipelined")
    p0.record(stream)
    pipelined(0, args.steps)
    p1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    wall_p = time.perf_counter() - wall0_p
    clk = clocks.stop()
    wrs.check_status(status)
    # untimed: the pipelined loop's last view equals a trace of a fresh build of that frame
    g_last = (args.steps - 1) % n_groups
    fb, fs = wrs.build_lbvh(wrs.unproject(*groups[g_last][:3]), leaf, layout=layout)
    ref0 = wrs.trace(fb, fs, groups[g_last][3][0], params)
    if not torch.equal(ref0.view(torch.int32), outs[0].view(torch.int32)):
        raise RuntimeError("pipelined step: the last view differs from a sequential build's")
    del fb, fs, ref0

    step_ms = [ev[0].elapsed_time(ev[-1]) for ev in events]
    up_ms = [ev[0].elapsed_time(ev[1]) for ev in events]
    bv_ms = [ev[1].elapsed_time(ev[2]) for ev in events]
    tr_ms = [ev[2 + f].elapsed_time(ev[3 + f]) for ev in events for f in range(FRAMES_PER_IMAGE)]
    seq_ms = max_over_ranks(sum(step_ms))
    seq_value = reps.whole_job_rate(args.steps * rays_per_step, seq_ms * 1e-3) / 1e6
    total_ms = max_over_ranks(p0.elapsed_time(p1))
    value = reps.whole_job_rate(args.steps * rays_per_step, total_ms * 1e-3) / 1e6
    trace_ms = statistics.mean(tr_ms)

    peaks, peak_src = measured_peaks()
    bpr = trace_bytes_per_ray(cnt_tot, rays_counted, width)
    fpr = trace_flops_per_ray(cnt_tot, rays_counted)
    bytes_launch = bpr * npix_c
    achieved = bytes_launch / (trace_ms * 1e-3) / 1e9
    # profiled per-launch figures (a few launches over poses spread across the set) scaled to the
    # timed poses by node visits per launch (the traversal's unit of work)
    nodes_profiled = profiled("node_visits_per_launch")
    pscale = (cnt_tot["nodes"] / (rays_counted / npix_c)) / nodes_profiled if nodes_profiled else None
    traffic = profiled_traffic()
    if traffic is not None and pscale is not None:
        traffic *= pscale
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "kernel": ["k_trace", "k_trace_pr", "k_trace_packet"][sched],
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                "bytes_per_ray": bpr, "flops_per_ray": fpr,
                "fp32_tflops_achieved": fpr * npix_c / (trace_ms * 1e-3) / 1e12,
                "counts_per_ray": {k: v / rays_counted for k, v in cnt_tot.items()},
                "traffic_source": "not measured in this run: dram__bytes_read.sum + "
                                  "dram__bytes_write.sum per launch from the committed ncu summary "
                                  "profiles/trace_large_1080p_bench_poses.md (4 launches over "
                                  "depth-image groups spread across the pose set), scaled by "
                                  "this run's counted node visits per launch over the profiled "
                                  "launches' (profile_scale); reported only while its recorded "
                                  "kernel digest matches the current trace source (else null)",
                "profile_scale": pscale}
    if traffic is not None:
        # what DRAM really moves per launch, as a rate against the same peak
        roofline["dram_frac"] = traffic / (trace_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]
    if roofline["frac"] > 1.0:
        roofline["frac_note"] = (
            "above 1: the counted bytes (the node and splat records each ray reads, counted by "
            "wrs_trace_count) are mostly re-read from L1 (73 % hit under ncu) and L2, not from "
            "DRAM; DRAM moves `traffic` bytes per launch (dram_frac of the HBM rate); against the "
            "L2-resident copy rate the counted bytes reach l2_frac; the binding limit is "
            "instruction issue on the ALU pipe (`issue`)")

    lbvh_bps = lbvh_bytes_per_splat(leaf, layout == wrs.LBVH_FULL)
    lbvh_gbs = lbvh_bps * statistics.mean(n_splats) / (statistics.mean(bv_ms) * 1e-3) / 1e9
    lbvh_roof = {"bound": "hbm", "bytes_per_splat": lbvh_bps, "achieved": lbvh_gbs,
                 "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": lbvh_gbs / peaks["hbm_gbs"],
                 "gsplat_s": statistics.mean(n_splats) / (statistics.mean(bv_ms) * 1e-3) / 1e9,
                 "note": "algorithmic bytes of the build's 16 kernels (lbvh_bytes_per_splat) over "
                         "the sequential loop's LBVH time; the build is latency-bound (the "
                         "refit's climb, Karras' divergent searches, the sort's scatter), not "
                         "bandwidth-bound"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(W, statistics.mean(n_splats), {
                "leaf_size": leaf, "k_chunk": kc,
                "block": launched_block(block, kc, width, sched),
                "autotuned": not args.no_autotune,
                "schedule": SCHEDULE_NAMES[sched],
                "bvh_width": width,
                "l2": ("not flushed: every step reads the next of 15 server images (622 MB in "
                       "rotation, so no step's input is left in L2) and rebuilds a 0.4 GB tree; "
                       "the sequential split below flushes L2 (256 MiB write) before every step "
                       "outside its events"),
                "pipeline": ("two buffer slots: frame g+1's unproject and LBVH build run on a "
                             "build stream of higher priority while frame g's 4 client views "
                             "trace; every step does the whole path, timed from the first "
                             "build to the last trace"),
                "lbvh_launch": "one CUDA graph of its 16 kernels, replayed every step",
                "lbvh_layout": ("4-wide nodes only (no binary records inside a refit block)"
                                if layout == wrs.LBVH_WIDE else "binary records and 4-wide nodes"),
                "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}),
            "sequential": {"mrays_s": seq_value, "ms_per_step": seq_ms / args.steps,
                           "wall_s": wall,
                           "note": "the same steps one after another on one stream, each "
                                   "bracketed by its own events after an L2 flush; the stage "
                                   "split below is from this loop"},
            "lbvh_ms": statistics.mean(bv_ms), "lbvh_roofline": lbvh_roof,
            "unproject_ms": statistics.mean(up_ms),
            "trace_ms": trace_ms, "trace_mrays_s": npix_c / (trace_ms * 1e-3) / 1e6,
            "wall_s_timed_region": wall_p,
            "paper_context": {"hardware": "RTX 2080", "lbvh_ms_623k": 11, "compact_ms": 23,
                              "mrays_s_1024sq_derived": [306, 289, 297, 240, 428]},
            "roofline": roofline, "gpu_launches": launches_per_step * args.steps}  # pipelined loop
    if clk:
        line["clocks"] = clk
    # the bound the profile shows: instruction issue.  Warp instructions per launch (ncu, same
    # kernel source) over the live launch time, against 148 SMs x 4 schedulers x 1 instruction
    # per cycle at the sampled SM clock
    winst = profiled("warp_instructions_per_launch")
    if winst is not None and pscale is not None:
        winst *= pscale
    profiled_launch = sched == 0 and width == 4 and kc == 1 and leaf == 1  # the captured launch
    fma = fma_rates(wrs, torch)
    line["roofline"]["fp32_peak_tflops_measured"] = fma["tflops"]
    # the same counted bytes against the L2 copy rate: rays re-read the upper tree levels and
    # neighbouring splats from L2/L1, so this is the cache-side bound (own streaming copy)
    cr = copy_rates(wrs, torch)
    line["roofline"]["own_copy_gbs"] = cr
    line["roofline"]["l2_frac"] = achieved / cr["l2_gbs"]
    alu = profiled("alu_pipe_warp_instructions_per_launch")
    alu_view = None
    if alu is not None and pscale is not None and clk and clk.get("sm_mhz"):
        # the ALU pipe (integer, compare, select, min/max) takes a warp instruction every second
        # cycle per scheduler: its share of the launch's cycles
        alu *= pscale
        alu_view = {"warp_instructions_per_launch": alu,
                    "frac": alu * 2 / (148 * 4 * clk["sm_mhz"] * 1e6 * trace_ms * 1e-3),
                    "note": "ALU-pipe warp instructions (profiled, scaled) x 2 cycles over the "
                            "launch's scheduler cycles at the sampled SM clock"}
    if winst is not None and profiled_launch and clk and clk.get("sm_mhz"):
        peak_gi = 148 * 4 * clk["sm_mhz"] * 1e6 / 1e9
        ach_gi = winst / (trace_ms * 1e-3) / 1e9
        line["roofline"]["issue"] = {"source": "warp instructions per launch from the committed "
                                               "ncu summary profiles/trace_large_1080p_bench_poses.md "
                                               "(digest-matched), scaled by node visits to the "
                                               "timed poses (profile_scale); launch time and SM "
                                               "clock live from this run",
                                     "warp_instructions_per_launch": winst,
                                     "achieved_ginst_s": ach_gi, "peak_ginst_s": peak_gi,
                                     "frac": ach_gi / peak_gi,
                                     "peak_ginst_s_measured": fma["ginst_s"],
                                     "frac_of_measured": ach_gi / fma["ginst_s"],
                                     "alu_pipe": alu_view,
                                     "measured_by": "wrs_fma_peak: FFMA warp instructions per "
                                                    "second of an FMA-only kernel, one wave of "
                                                    "8 x 256 threads per SM",
                                     "note": "the kernel's binding limit (ALU pipe 71 %, issue "
                                             "68-69 % under ncu); the hbm entry is the "
                                             "counted-bytes roofline"}

    if not args.no_extras:
        extras(line, args, wrs, autotune, synth, torch, groups, params, leaf, rank, world, barrier,
               max_over_ranks, large_vol=vol)
    if rank == 0:
        print(json.dumps(line), flush=True)
    reps.close()


def run_case(a, wrs, torch):
    """One workload of the hot path once, with few launches, for ncu captures: the server image
    from the GPU ray caster (volume freed afterwards), unproject, LBVH build and client traces,
    each stage in its own NVTX range; prints the CUDA event times as one JSON line.

    large/mid/tiny: ``--groups g0,g1,..`` ray-casts the server image of each depth-image group of
    the benchmark (pose 4g) and traces ``--frames`` of its client poses, so that a few launches
    sample poses spread over the set; without it, the server camera and the first ``--frames``
    poses.  diff: two forward + backward steps of the 8 views of the differentiation workload
    (one launch each way per step; the forward records the hit lists and the adjoint runs from
    them, or with ``--retraverse`` the adjoint traces every ray again).  batched: the first ``--sessions`` of the multi-session
    workload, two launches of wrs_trace_batched (the second is the one to profile)."""
    import synth
    if a.case == "diff":
        return _case_diff(a, wrs, torch, synth)
    if a.case == "batched":
        return _case_batched(a, wrs, torch, synth)
    W = {"tiny": synth.TINY, "mid": synth.MID, "large": synth.LARGE}[a.case]
    dev = torch.device("cuda")
    vol = torch.from_numpy(W.volume()).to(dev)
    tf = torch.from_numpy(synth.tf_ramp()).to(dev)
    poses = W.client_poses()
    plan = []  # (server camera, client cameras)
    if a.groups:
        for g in (int(x) for x in a.groups.split(",")):
            srv = poses[FRAMES_PER_IMAGE * g].with_size(W.server_w, W.server_h)
            plan.append((srv, [poses[FRAMES_PER_IMAGE * g + f] for f in range(a.frames)]))
    else:
        plan.append((W.server_cam(), poses[: a.frames]))
    images = [wrs.raycast_volume(vol, tf, srv) for srv, _ in plan]
    del vol
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    params = wrs.TraceParams(max_hits=a.max_hits, k_chunk=a.k, block=a.block, schedule=a.schedule,
                             width=a.width)
    layout = {"auto": wrs.tree_layout(params), "full": wrs.LBVH_FULL,
              "wide": wrs.LBVH_WIDE}[a.layout]
    st = wrs.new_status()
    out = torch.empty(W.client_h, W.client_w, 4, device=dev)
    res = {"workload": a.case, "groups": a.groups or None, "layout": layout, "splats": [],
           "unproject_ms": [], "lbvh_ms": [], "trace_ms": []}
    for (srv, clis), (rgba, depth) in zip(plan, images):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 + len(clis))]
        ev[0].record()
        torch.cuda.nvtx.range_push("unproject")
        sp = wrs.unproject(rgba, depth, srv)
        torch.cuda.nvtx.range_pop()
        ev[1].record()
        torch.cuda.nvtx.range_push("lbvh")
        bvh, srt = wrs.build_lbvh(sp, a.leaf, layout=layout)
        torch.cuda.nvtx.range_pop()
        ev[2].record()
        for f, c in enumerate(clis):
            torch.cuda.nvtx.range_push(f"trace{f}")
            wrs.trace(bvh, srt, wrs.make_camera(c), params, out=out, status=st)
            torch.cuda.nvtx.range_pop()
            ev[3 + f].record()
        torch.cuda.synchronize()
        res["splats"].append(sp.count())
        res["unproject_ms"].append(ev[0].elapsed_time(ev[1]))
        res["lbvh_ms"].append(ev[1].elapsed_time(ev[2]))
        res["trace_ms"] += [ev[2 + f].elapsed_time(ev[3 + f]) for f in range(len(clis))]
        # counted work of each traced launch (k_trace_count, after the timed launches), so that
        # profiled figures of these launches can be scaled to other poses by node visits
        res.setdefault("node_visits", []).extend(
            wrs.trace_count(bvh, srt, wrs.make_camera(c), params)["nodes"] for c in clis)
        del sp, bvh, srt
    wrs.check_status(st)
    res["device_bytes_allocated"] = torch.cuda.memory_allocated()
    print(json.dumps(res))


def _case_diff(a, wrs, torch, synth):
    D = synth.DIFF
    dev = torch.device("cuda")
    tf = torch.from_numpy(synth.tf_ramp()).to(dev)
    vol = synth.gaussian_volume_device(D.vol_n, D.vol_param, D.seed)
    srv = D.server_cam()
    rgba, depth = wrs.raycast_volume(vol, tf, srv)
    views = D.client_poses()
    target = torch.stack([wrs.raycast_volume(vol, tf, v)[0] for v in views])
    del vol
    sp = wrs.unproject(rgba, depth, srv)
    n = sp.count()
    col = sp.rgba[:n].clone().requires_grad_(True)
    opa = torch.ones(n, device=dev, requires_grad=True)
    scl = torch.ones(n, device=dev, requires_grad=True)
    params = wrs.TraceParams(0, 1e-5, 0.25, a.k, 128, a.schedule, 4)
    ms = []
    for _ in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        loss = torch.nn.functional.mse_loss(
            wrs.render_views(sp, views, col, opa, scl, params, a.leaf,
                             record_hits=0 if a.retraverse else None), target)
        loss.backward()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    print(json.dumps({"workload": "diff", "splats": n, "views": len(views),
                      "adjoint": "re-traversal" if a.retraverse else "recorded hit lists",
                      "fwd_bwd_ms": ms, "loss": float(loss.detach())}))


def _case_batched(a, wrs, torch, synth):
    dev = torch.device("cuda")
    tf = torch.from_numpy(synth.tf_ramp()).to(dev)
    sess = []
    n_splats = 0
    for s, (size, srv, cli) in enumerate(synth.batched_sessions(64, seed=4000)[: a.sessions]):
        vol = synth.gaussian_volume_device(256, 64, 4000 + s)
        rgba, depth = wrs.raycast_volume(vol, tf, srv)
        del vol
        sp = wrs.unproject(rgba, depth, srv)
        bvh, srt = wrs.build_lbvh(sp, a.leaf)
        n_splats += sp.count()
        sess.append((bvh, srt, cli))
        del sp
    batch = wrs.Batch(sess)
    params = wrs.TraceParams(max_hits=a.max_hits, k_chunk=a.k, schedule=a.schedule, width=a.width)
    st = wrs.new_status()
    ms = []
    for _ in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.cuda.nvtx.range_push("batched")
        wrs.trace_batched(batch, params, status=st)
        torch.cuda.nvtx.range_pop()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    wrs.check_status(st)
    rays = sum(c.width * c.height for _, _, c in sess)
    print(json.dumps({"workload": "batched", "sessions": len(sess), "splats": n_splats,
                      "rays": rays, "trace_batched_ms": ms,
                      "device_bytes_allocated": torch.cuda.memory_allocated()}))


def size_scaling(wrs, torch):
    """Unproject and LBVH (leaf 1) over server frames of 512^2 .. 4096^2 pixels of the large
    workload's volume, and the trace (one thread per pixel and persistent, K 1 and 2, 4-wide
    nodes) of the 1080p frame's splats into clients of 256^2 .. 4096^2 at one pose.  CUDA events,
    warm L2, mean of 10 launches after 3."""
    import synth

    def tms(fn, reps=10, warm=3):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    dev = torch.device("cuda")
    W = synth.LARGE
    vol = torch.from_numpy(W.volume()).to(dev)
    tf = torch.from_numpy(synth.tf_ramp()).to(dev)
    base, pose = W.server_cam(), W.client_poses(2)[1]
    builds, traces = [], []
    for (w, h) in ((512, 512), (1024, 1024), (1920, 1080), (2048, 2048), (3840, 2160),
                   (4096, 4096)):
        srv = base.with_size(w, h)
        r, d = wrs.raycast_volume(vol, tf, srv)
        sp = wrs.unproject(r, d, srv)
        scr = torch.empty(max(wrs.unproject_scratch_bytes(w, h), 256), dtype=torch.uint8,
                          device=dev)
        up = tms(lambda: wrs.unproject(r, d, srv, out=sp, scratch=scr))
        # the traces below walk the 4-wide nodes: the 4-wide-only layout, as in the benchmark
        bvh = wrs.LBVH(w * h, 1, layout=wrs.LBVH_WIDE)
        srt = wrs.SplatBuffers(w * h, sorted=True)
        bs = torch.empty(wrs.lbvh_scratch_bytes(w * h, 1), dtype=torch.uint8, device=dev)
        lb = tms(lambda: wrs.build_lbvh(sp, 1, bvh=bvh, sorted=srt, scratch=bs))
        n = sp.count()
        builds.append({"server": [w, h], "splats": n, "unproject_ms": up, "lbvh_ms": lb,
                       "lbvh_gsplat_s": n / lb / 1e6})
        if (w, h) == (1920, 1080):
            for (cw, ch) in ((256, 256), (512, 512), (1024, 1024), (1920, 1080), (2048, 2048),
                             (3840, 2160), (4096, 4096)):
                cli = wrs.make_camera(pose.with_size(cw, ch))
                out = torch.empty(ch, cw, 4, device=dev)
                row = {"client": [cw, ch]}
                for sched in (0, 1):
                    for k in (1, 2):
                        p = wrs.TraceParams(0, 1e-5, 0.0, k, 128, sched, 4)
                        t = tms(lambda: wrs.trace(bvh, srt, cli, p, out=out))
                        row[f"{SCHEDULE_NAMES[sched]}, K {k}: Mrays/s"] = cw * ch / t / 1e3
                traces.append(row)
        del sp, bvh, srt, bs, scr, r, d
        torch.cuda.empty_cache()
    return {"size_scaling": {"build": builds, "trace_on_1080p_frame": traces,
                             "workload": W.name, "leaf_size": 1, "lbvh_layout": "4-wide nodes only",
                             "l2": "warm"}}


def fma_rates(wrs, torch, iters=2000, reps=5):
    """Measured binary32 FMA throughput (TFLOP/s) and FFMA warp-instruction rate (G/s) of this
    GPU: wrs_fma_peak on 8 blocks of 256 threads per SM, median of reps (CUDA events)."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks = sms * 8
    out = torch.empty(blocks, dtype=torch.float32, device="cuda")
    flops = 0.0
    for _ in range(2):
        flops = wrs.fma_peak(blocks, iters, out=out)
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        wrs.fma_peak(blocks, iters, out=out)
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b) * 1e-3)
    t = statistics.median(ts)
    return {"tflops": flops / t / 1e12, "ginst_s": flops / 2 / 32 / t / 1e9}


def copy_rates(wrs, torch, reps=5):
    """Own copy-rate measurements (GB/s, bytes read + written): wrs_stream_copy over 1 GiB
    buffers (HBM) and, 100 times over in one launch, over 16 MiB buffers that stay in L2."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = {}
    for name, nbytes, inner in (("hbm_gbs", 1 << 30, 1), ("l2_gbs", 16 << 20, 100)):
        a = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        b = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        a.fill_(1)
        for _ in range(3):
            wrs.stream_copy(b, a, sms * 8, inner)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            wrs.stream_copy(b, a, sms * 8, inner)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        out[name] = 2 * nbytes * inner / statistics.median(ts) / 1e9
        del a, b
    return out


def link_rates(torch, nbytes, reps=5):
    """Pinned host <-> device copy rates in GB/s (CUDA events, median of reps, one direction at
    a time)."""
    host = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    dev = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    out = {}
    for name, dst, src in (("h2d_gbs", dev, host), ("d2h_gbs", host, dev)):
        dst.copy_(src, non_blocking=True)
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            dst.copy_(src, non_blocking=True)
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        out[name] = nbytes / (statistics.median(ts) * 1e-3) / 1e9
    del host, dev
    return out


def _time_ms(torch, fn, reps, warm=3):
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


def extras(line, args, wrs, autotune, synth, torch, groups, params, leaf, rank, world, barrier,
           max_over_ranks, large_vol=None):
    dev = torch.device("cuda")
    W = synth.LARGE
    npix_s = W.server_w * W.server_h
    npix_c = W.client_w * W.client_h
    # ---------------- end to end through host buffers ------------------------------------------
    # The client pipeline (WarpingClient): every step copies a server frame from pinned host
    # memory, rebuilds splats and LBVH, traces 4 views and copies each view back to pinned host
    # memory; the copies run on their own streams and overlap the GPU work of neighbouring
    # frames.  Timed by the host clock between two device synchronisations.
    from paper_2006_14726_b300.client import WarpingClient
    h_groups = [(g[0].cpu().pin_memory(), g[1].cpu().pin_memory(), g[2], g[3]) for g in groups[:4]]
    client = WarpingClient(W.server_w, W.server_h, W.client_w, W.client_h, params, leaf)

    def e2e_run(steps):
        prev = []
        for st in range(steps):
            hr, hd, srv_h, clis_h = h_groups[st % len(h_groups)]
            client.submit(hr, hd, srv_h)
            cur = [client.render(c) for c in clis_h]
            for tk in prev:  # collect the previous step's views while this step runs
                client.result(tk)
            prev = cur
        for tk in prev:
            client.result(tk)
    e2e_run(5)
    torch.cuda.synchronize()
    steps = 200
    barrier()
    t0 = time.perf_counter()
    e2e_run(steps)
    torch.cuda.synchronize()
    ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / steps)
    wrs.check_status(client.status)
    hr0, hd0 = h_groups[0][0], h_groups[0][1]
    h2d_bytes = int(hr0.numel() * 4 + hd0.numel() * 4)
    d2h_bytes = int(FRAMES_PER_IMAGE * W.client_w * W.client_h * 16)
    del client
    # the host link's own copy rates (pinned, one direction at a time): with the step's device
    # time they bound the end-to-end step from below
    link = link_rates(torch, 128 << 20)
    bound_ms = max(line["ms_per_step"], h2d_bytes / (link["h2d_gbs"] * 1e6),
                   d2h_bytes / (link["d2h_gbs"] * 1e6))
    line["e2e"] = {"value": world * FRAMES_PER_IMAGE * npix_c / (ms * 1e-3) / 1e6, "unit": UNIT,
                   "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": d2h_bytes,
                   "ms_per_step": ms, "steps": steps,
                   "link_gbs": link, "bound_ms_per_step": bound_ms,
                   "frac_of_bound": bound_ms / ms,
                   "bound": "max(device step, h2d bytes / h2d rate, d2h bytes / d2h rate)",
                   "path": "WarpingClient: pinned host frame -> device (copy stream), unproject "
                           "and LBVH (build stream, higher priority), 4 traces (trace stream), 4 "
                           "images -> pinned host (copy stream); copies and the next frame's "
                           "build overlap neighbouring frames' traces; host clock"}

    # ---------------- batched: 64 sessions, one launch in a CUDA graph ------------------------
    sessions = synth.batched_sessions(64, seed=4000 + 1000 * rank)
    tfd = torch.from_numpy(synth.tf_ramp()).to(dev)
    sess = []
    n_total_splats = 0
    for s, (size, srv_s, cli_s) in enumerate(sessions):
        vol = synth.gaussian_volume_device(256, 64, 4000 + s + 1000 * rank)
        rgba_s, depth_s = wrs.raycast_volume(vol, tfd, srv_s)
        del vol
        sp = wrs.unproject(rgba_s, depth_s, srv_s)
        b, so = wrs.build_lbvh(sp, leaf)
        n_total_splats += sp.count()
        sess.append((b, so, cli_s))
        del sp
    batch = wrs.Batch(sess)
    bt = autotune.tune_batched(batch, params)
    bparams = wrs.TraceParams(0, 1e-5, 0.0, bt["k_chunk"], bt["block"], bt["schedule"], bt["width"])
    outs = [torch.empty(c.height, c.width, 4, device=dev) for _, _, c in sess]
    seq_cams = [wrs.make_camera(c) for _, _, c in sess]

    def sequential():
        for (b, so, _), c, o in zip(sess, seq_cams, outs):
            wrs.trace(b, so, c, params, out=o)
    # the same 64 calls with the batched launch's own knobs: K, block, node width, and each
    # session's schedule as the one launch traces it -- what one launch gains by itself
    own = [wrs.TraceParams(0, 1e-5, 0.0, bt["k_chunk"], bt["block"],
                           batch.schedules[i] if bt["schedule"] == wrs.SCHEDULE_PER_SESSION
                           else bt["schedule"], bt["width"]) for i in range(len(sess))]

    def sequential_own():
        for (b, so, _), c, o, p_s in zip(sess, seq_cams, outs, own):
            wrs.trace(b, so, c, p_s, out=o)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        wrs.trace_batched(batch, bparams)  # warm (caches the launch shape outside capture)
        with torch.cuda.graph(g, stream=side):
            wrs.trace_batched(batch, bparams)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    rays = sum(c.width * c.height for _, _, c in sess)
    barrier()
    ms_graph = max_over_ranks(_time_ms(torch, g.replay, 10))
    ms_seq = max_over_ranks(_time_ms(torch, sequential, 10))
    ms_own = max_over_ranks(_time_ms(torch, sequential_own, 10))
    line["batched"] = {"sessions": len(sess), "rays_per_launch": rays,
                       "splats_total": n_total_splats,
                       "server_sizes": sorted({int(s[0]) for s in sessions}),
                       "one_launch_graph_mrays_s": world * rays / (ms_graph * 1e-3) / 1e6,
                       "sequential_mrays_s": world * rays / (ms_seq * 1e-3) / 1e6,
                       "sequential_same_knobs_mrays_s": world * rays / (ms_own * 1e-3) / 1e6,
                       "one_launch_ms": ms_graph, "sequential_ms": ms_seq,
                       "sequential_same_knobs_ms": ms_own,
                       "sequential_note": "sequential: 64 wrs_trace calls with the large "
                                          "workload's launch; sequential_same_knobs: the same "
                                          "calls with the one launch's K, block, node width and "
                                          "each session's own schedule, so the gain of one "
                                          "launch alone is one_launch vs sequential_same_knobs",
                       "k_chunk": bt["k_chunk"], "block": bt["block"], "bvh_width": bt["width"],
                       "schedule": (SCHEDULE_NAMES[bt["schedule"]] if bt["schedule"] < 3 else
                                    "per session: packet for the {} sessions with >= {:g} "
                                    "client pixels per splat, one thread per pixel for the other "
                                    "{}".format(sum(v == wrs.SCHEDULE_PACKET for v in batch.schedules),
                                                wrs.SPARSE_PIXELS_PER_SPLAT,
                                                sum(v != wrs.SCHEDULE_PACKET for v in batch.schedules))),
                       "leaf_size": leaf}
    del sess, batch, outs, g

    # ---------------- accumulation over a window of server frames (one LBVH over all) -----------
    # The union of several frames has several times the hits per ray of one frame, so the launch
    # is tuned again on the window (untimed).
    F_WIN = 4
    probe = wrs.FrameWindow(F_WIN, W.server_w, W.server_h, decay=0.9)
    for g_i in range(F_WIN):
        probe.push(*groups[g_i][:3])
    at = autotune.tune_trace(probe.splats, groups[F_WIN][3], use_cache=False,
                             build_weight=1.0 / FRAMES_PER_IMAGE)
    del probe
    aparams = wrs.TraceParams(max_hits=0, t_stop=1e-5, k_chunk=at["k_chunk"], block=at["block"],
                              schedule=at["schedule"], width=at["width"])
    # two copies of the window's set: the next frame's push (unproject of the 4 frames + LBVH) on
    # a build stream of higher priority overlaps this frame's 4 traces
    win = wrs.FrameWindow(F_WIN, W.server_w, W.server_h, decay=0.9, leaf_size=at["leaf"],
                          layout=tree_layout(wrs, at["width"], at["schedule"]), slots=2)
    abuild = torch.cuda.Stream(priority=-1)
    for g_i in range(F_WIN):
        win.push(*groups[g_i][:3])
    outs = [torch.empty(W.client_h, W.client_w, 4, device=dev) for _ in range(FRAMES_PER_IMAGE)]
    nxt = [F_WIN]

    def acc_step():
        rgba_a, depth_a, srv_a, clis_a = groups[nxt[0] % len(groups)]
        nxt[0] += 1
        win.push(rgba_a, depth_a, srv_a, stream=abuild)
        for f in range(FRAMES_PER_IMAGE):
            win.trace(clis_a[f], aparams, out=outs[f])

    def acc_time(reps, warm=3):
        for _ in range(warm):
            acc_step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        abuild.wait_event(e0)  # the first timed push starts inside the timed region
        for _ in range(reps):
            acc_step()
        e1.record()  # after the last traces, which waited for the last push
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    barrier()
    ms_acc = max_over_ranks(acc_time(10))
    ms_rebuild = max_over_ranks(_time_ms(torch, win.rebuild, 10))
    # the 4 traces alone, over 4 more steps (each push on this stream, then the 4 views between
    # two events): windows of the same kind as the timed loop's
    tr = []
    for _ in range(4):
        rgba_a, depth_a, srv_a, clis_a = groups[nxt[0] % len(groups)]
        nxt[0] += 1
        win.push(rgba_a, depth_a, srv_a)
        ta, tb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ta.record()
        for f in range(FRAMES_PER_IMAGE):
            win.trace(clis_a[f], aparams, out=outs[f])
        tb.record()
        torch.cuda.synchronize()
        tr.append(ta.elapsed_time(tb))
    ms_tr = max_over_ranks(statistics.mean(tr))
    wrs.check_status(win.status)
    line["accumulate"] = {"frames": F_WIN, "decay": 0.9, "splats": win.splats.count(),
                          "client_frames_per_server_frame": FRAMES_PER_IMAGE,
                          "mrays_s": world * FRAMES_PER_IMAGE * npix_c / (ms_acc * 1e-3) / 1e6,
                          "ms_per_step": ms_acc, "rebuild_ms": ms_rebuild,
                          "trace_ms": ms_tr / FRAMES_PER_IMAGE,
                          "leaf_size": at["leaf"], "k_chunk": at["k_chunk"],
                          "block": launched_block(at["block"], at["k_chunk"], at["width"],
                                                  at["schedule"]),
                          "schedule": SCHEDULE_NAMES[at["schedule"]], "bvh_width": at["width"],
                          "pipeline": "two copies of the window: the next frame's push on a "
                                      "build stream of higher priority overlaps the 4 traces",
                          "note": "step = push one 1080p server frame into the window of the 4 "
                                  "newest (4 unprojections into one set + LBVH over about 8 M "
                                  "splats) + 4 client traces of the union"}
    del win, outs

    # ---------------- mid workload: trace only, 1024^2 client, 262 k splats (median over poses) --
    M = synth.MID
    vol_m = synth.gaussian_volume_device(M.vol_n, M.vol_param, M.seed + rank)
    srv_m = M.server_cam()
    rgba_m, depth_m = wrs.raycast_volume(vol_m, torch.from_numpy(synth.tf_ramp()).to(dev), srv_m)
    del vol_m
    sp_m = wrs.unproject(rgba_m, depth_m, srv_m)
    cams_m = [wrs.make_camera(c) for c in M.client_poses(seed_offset=rank)]
    # the launch tuned on this workload (a trace-only number: no build share in the score)
    tm = autotune.tune_trace(sp_m, cams_m[:4], use_cache=False) if not args.no_autotune else \
        {"leaf": leaf, "k_chunk": params.k_chunk, "block": params.block,
         "schedule": params.schedule, "width": params.width}
    mparams = wrs.TraceParams(max_hits=0, t_stop=1e-5, k_chunk=tm["k_chunk"], block=tm["block"],
                              schedule=tm["schedule"], width=tm["width"])
    bvh_m, srt_m = wrs.build_lbvh(sp_m, tm["leaf"],
                                  layout=tree_layout(wrs, tm["width"], tm["schedule"]))
    out_m = torch.empty(M.client_h, M.client_w, 4, device=dev)
    per_pose = []
    for c in cams_m:
        per_pose.append(_time_ms(torch, lambda: wrs.trace(bvh_m, srt_m, c, mparams, out=out_m), 10))
    ms_m = max_over_ranks(statistics.median(per_pose))
    line["mid"] = {"splats": sp_m.count(), "client": [M.client_w, M.client_h], "poses": len(cams_m),
                   "trace_ms_median": ms_m,
                   "trace_mrays_s": world * M.client_w * M.client_h / (ms_m * 1e-3) / 1e6,
                   "launch": {"leaf_size": tm["leaf"], "k_chunk": tm["k_chunk"],
                              "schedule": SCHEDULE_NAMES[tm["schedule"]], "bvh_width": tm["width"]},
                   "lbvh_ms": max_over_ranks(_time_ms(torch, lambda: wrs.build_lbvh(
                       sp_m, tm["leaf"], bvh=bvh_m, sorted=srt_m), 10))}
    if rank == 0 and world == 1:
        import oracle
        oracle.build()
        t, r, det = oracle_step_time(rgba_m.cpu().numpy(), depth_m.cpu().numpy(), srv_m,
                                     M.client_poses()[:2], ray_stride=8,
                                     threads=oracle.default_threads())
        line["mid"]["cpu_oracle_trace_mrays_s"] = r / det["trace_s_extrapolated"] / 1e6
        line["mid"]["cpu_oracle_bvh_s"] = det["bvh_s"]
    del sp_m, bvh_m, srt_m, out_m

    # ---------------- image quality, Fig. 3 as numbers: spheres vs fixed-size points ------------
    from paper_2006_14726_b300.quality import warp_quality
    if large_vol is not None:
        srv_q = groups[0][2]
        angles = (2.0, 5.0, 10.0, 20.0)
        clis_q = [synth.orbit(srv_q, (0.6, 0.8, 0.0), a) for a in angles]
        blobs = synth.gaussian_volume_device(256, 64, 2000)
        scenes = {"fourier_512_ramp_tf": (large_vol, synth.tf_ramp(), 3 ** 0.5 / 512),
                  "blobs_256_iso_tf": (blobs, synth.tf_iso(), 3 ** 0.5 / 256)}
        q = {"metric": "PSNR dB vs the ray caster at the client pose (all four premultiplied "
                       "channels)", "server_and_client": [srv_q.width, srv_q.height],
             "angles_deg": list(angles)}
        for name, (v, tf_np, vd) in scenes.items():
            rows = warp_quality(v, torch.from_numpy(tf_np).to(dev), srv_q, clis_q, voxel_diag=vd,
                                interval_chain=8)
            q[name] = [{k: (round(x, 3) if x is not None else None) for k, x in r.items()}
                       for r in rows]
        # the server's depth rule (first hit, max contribution, accumulated opacity, max
        # gradient: Fig. 3 uses a gradient heuristic) on the iso scene, at 10 and 20 degrees
        names = {0: "first_hit", 1: "max_contribution", 2: "accumulated_0.5", 3: "max_gradient"}
        q["heuristics_blobs_256_iso_tf"] = {}
        for hh, nm in names.items():
            rows = warp_quality(blobs, torch.from_numpy(synth.tf_iso()).to(dev), srv_q, clis_q[2:],
                                point_sizes=(2, 3), max_hits=(0,), voxel_diag=3 ** 0.5 / 256,
                                heuristic=hh)
            q["heuristics_blobs_256_iso_tf"][nm] = [
                {k: (round(x, 3) if x is not None else None) for k, x in r.items()} for r in rows]
        del blobs
        # cost of the two warps on the same 1080p frame (one client view)
        sp_q = wrs.unproject(groups[0][0], groups[0][1], srv_q)
        bvh_q, srt_q = wrs.build_lbvh(sp_q, leaf)
        out_q = torch.empty(W.client_h, W.client_w, 4, device=dev)
        psc = torch.empty(wrs.point_splat_scratch_bytes(W.client_w, W.client_h), dtype=torch.uint8,
                          device=dev)
        c_q = wrs.make_camera(clis_q[-1])
        q["ms_per_view"] = {
            "spheres_trace": _time_ms(torch, lambda: wrs.trace(bvh_q, srt_q, c_q, params, out=out_q), 20),
            "points_1px": _time_ms(torch, lambda: wrs.point_splat(sp_q, c_q, 1, out=out_q, scratch=psc), 20),
            "points_3px": _time_ms(torch, lambda: wrs.point_splat(sp_q, c_q, 3, out=out_q, scratch=psc), 20)}
        line["quality"] = q

        # ---------------- 64-bit quantised splat stream (12 B per splat instead of 36) ----------
        from paper_2006_14726_b300.quality import psnr
        r_max = float(sp_q.pos_r[:sp_q.count(), 3].max())
        codec = wrs.make_codec((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), r_max)
        rgba0, depth0 = groups[0][0], groups[0][1]
        enc = wrs.unproject_encode(rgba0, depth0, srv_q, codec)
        dec = wrs.decode_splats(enc, codec)
        bvh_d, srt_d = wrs.build_lbvh(dec, leaf)
        ref_img = wrs.trace(bvh_q, srt_q, c_q, params)
        dec_img = wrs.trace(bvh_d, srt_d, c_q, params)
        usc = torch.empty(wrs.unproject_scratch_bytes(W.server_w, W.server_h), dtype=torch.uint8,
                          device=dev)
        line["codec"] = {
            "bytes_per_splat": 12, "float_bytes_per_splat": 36, "splats": enc.count(),
            "stream_mb": enc.nbytes() / 1e6,
            "unproject_encode_ms": _time_ms(torch, lambda: wrs.unproject_encode(
                rgba0, depth0, srv_q, codec, out=enc, scratch=usc), 20),
            "unproject_float_ms": _time_ms(torch, lambda: wrs.unproject(
                rgba0, depth0, srv_q, out=sp_q, scratch=usc), 20),
            "decode_ms": _time_ms(torch, lambda: wrs.decode_splats(enc, codec, out=dec), 20),
            "psnr_decoded_vs_float_view_db": psnr(dec_img, ref_img),
            "max_abs_decoded_vs_float_view": float((dec_img - ref_img).abs().max()),
            "box": "unit cube (the volume's bounds)", "r_max": r_max}
        del sp_q, bvh_q, srt_q, out_q, psc, enc, dec, bvh_d, srt_d

    # ---------------- forward and forward+backward (differentiable renderer) -------------------
    D = synth.DIFF
    vol_np = D.volume(seed_offset=rank)
    vol = torch.from_numpy(vol_np).to(dev)
    srv_d = D.server_cam()
    rgba_d, depth_d = wrs.raycast_volume(vol, tfd, srv_d)
    views = D.client_poses(seed_offset=rank)
    # reference views of the fit (untimed): the oracle's volume ray caster (binary64
    # compositing) on one GPU; with several ranks each takes its own views from the GPU ray
    # caster instead, so that N ranks do not share the host cores for it
    if world == 1:
        targets, target_src = oracle_views(vol_np, synth.tf_ramp(), views), "binary64 oracle ray cast"
        targets = [t.to(dev) for t in targets]
    else:
        targets = [wrs.raycast_volume(vol, tfd, v)[0] for v in views]
        target_src = "GPU ray caster"
    del vol
    sp = wrs.unproject(rgba_d, depth_d, srv_d)
    n = sp.count()
    col = sp.rgba[:n].clone().requires_grad_(True)
    opa = torch.ones(n, device=dev, requires_grad=True)
    scl = torch.ones(n, device=dev, requires_grad=True)
    # all views of a step share one LBVH build (one radius scale per step) and run in one launch;
    # the backward pass, also one launch, accumulates every view's gradient in place
    target = torch.stack(targets)
    cfg = {}

    def fwd():
        with torch.no_grad():
            wrs.render_views(sp, views, col, opa, scl, cfg["p"], cfg["leaf"], record_hits=0)

    def loss_fn(record=None):
        return torch.nn.functional.mse_loss(
            wrs.render_views(sp, views, col, opa, scl, cfg["p"], cfg["leaf"], record_hits=record),
            target)

    def fwd_bwd():  # the forward pass records the hit lists, the adjoint runs from them
        loss_fn().backward()

    def fwd_bwd_retraverse():  # the adjoint re-traverses every ray
        loss_fn(0).backward()

    def graphed(step):
        """``step`` captured in a CUDA graph after three eager runs on a side stream; the
        gradients are cleared before the capture, so every replay writes them afresh."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(3):
                step()
        torch.cuda.current_stream().wait_stream(side)
        for t in (col, opa, scl):
            t.grad = None
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr):
            step()
        return gr

    # the launch of this workload (soft edges, several hits per ray, 512^2 views) is tuned on the
    # forward + backward step itself, replayed from a CUDA graph (GPU time; the eager step's host
    # issue time depends on the host): leaf size, K, and the per-pixel or packet schedule
    d_table = []
    for d_leaf in (1, 2):
        for d_k in (1, 2, 4):
            for d_sched in (0, 2):
                cfg["p"] = wrs.TraceParams(0, 1e-5, 0.25, d_k, 128, d_sched, 4)
                cfg["leaf"] = d_leaf
                gr = graphed(fwd_bwd)
                d_table.append((_time_ms(torch, gr.replay, 10), d_leaf, d_k, d_sched))
                del gr
                for t in (col, opa, scl):
                    t.grad = None
    _, d_leaf, d_k, d_sched = min(d_table)
    cfg["p"] = wrs.TraceParams(0, 1e-5, 0.25, d_k, 128, d_sched, 4)
    cfg["leaf"] = d_leaf
    barrier()
    ms_f = max_over_ranks(_time_ms(torch, fwd, 20))
    ms_fb = max_over_ranks(_time_ms(torch, fwd_bwd, 20))
    ms_fbr = max_over_ranks(_time_ms(torch, fwd_bwd_retraverse, 20))
    gr = graphed(fwd_bwd)
    ms_fb_g = max_over_ranks(_time_ms(torch, gr.replay, 20))
    del gr
    gr = graphed(fwd_bwd_retraverse)
    ms_fbr_g = max_over_ranks(_time_ms(torch, gr.replay, 20))
    del gr
    for t in (col, opa, scl):
        t.grad = None
    rays_d = sum(v.width * v.height for v in views)
    # one step of the radius fit (rebuild, trace, loss, adjoint, Adam), eager and replayed from a
    # CUDA graph; the timed steps are real steps of two throw-away fits
    from paper_2006_14726_b300.fit import GRAPH_WARMUP, RadiusFit
    fit_ms = {}
    for graphed in (False, True):
        fz = RadiusFit(sp, views, target, cfg["p"], cfg["leaf"], lr=1e-2, rgba=col.detach(),
                       opacity=opa.detach(), graph=graphed)
        fz.run(GRAPH_WARMUP + 2)
        fit_ms[graphed] = max_over_ranks(_time_ms(torch, fz._step_async, 20))
        del fz
    # fit the per-splat radius scales to the novel views: 200 graphed Adam steps, lr 1e-2,
    # checkpointed after step 100 and resumed from the checkpoint in a new fit object
    ck = os.path.join(tempfile.gettempdir(), f"wrs_radius_fit_rank{rank}.pt")
    t_fit = time.perf_counter()
    f1 = RadiusFit(sp, views, target, cfg["p"], cfg["leaf"], lr=1e-2, rgba=col.detach(),
                   opacity=opa.detach(), graph=True)
    f1.run(100, checkpoint=ck, every=100)
    f2 = RadiusFit(sp, views, target, cfg["p"], cfg["leaf"], lr=1e-2, rgba=col.detach(),
                   opacity=opa.detach(), graph=True)
    f2.load(ck)
    f2.run(100)
    fit_s = time.perf_counter() - t_fit
    os.remove(ck)
    curve = [(i, f2.losses[i]) for i in list(range(0, 200, 20)) + [199]]
    scl = f2.scale
    line["fwd_bwd"] = {"views": len(views), "splats": n, "client": [D.client_w, D.client_h],
                       "edge_softness": 0.25,
                       "launch": {"leaf_size": d_leaf, "k_chunk": d_k,
                                  "schedule": SCHEDULE_NAMES[d_sched], "bvh_width": 4,
                                  "tuned_on": "forward + backward step replayed from a CUDA "
                                              "graph"},
                       "forward_mrays_s": world * rays_d / (ms_f * 1e-3) / 1e6,
                       "forward_backward_mrays_s": world * rays_d / (ms_fb * 1e-3) / 1e6,
                       "forward_backward_retraverse_mrays_s": world * rays_d / (ms_fbr * 1e-3) / 1e6,
                       "forward_backward_graphed_mrays_s": world * rays_d / (ms_fb_g * 1e-3) / 1e6,
                       "forward_backward_retraverse_graphed_mrays_s":
                           world * rays_d / (ms_fbr_g * 1e-3) / 1e6,
                       "forward_ms_per_view": ms_f / len(views),
                       "forward_backward_ms_per_view": ms_fb / len(views),
                       "adjoint": "forward_backward: the forward launch records each ray's "
                                  "composited hits (16 per ray, the rest traced again) and the "
                                  "adjoint runs from them without traversal; "
                                  "forward_backward_retraverse: the adjoint traces every ray "
                                  "again (replay and re-gather)",
                       "fit_step_mrays_s": world * rays_d / (fit_ms[False] * 1e-3) / 1e6,
                       "fit_step_graphed_mrays_s": world * rays_d / (fit_ms[True] * 1e-3) / 1e6,
                       "fit_step_ms": fit_ms[False], "fit_step_graphed_ms": fit_ms[True],
                       "fit": {"steps": 200, "optimizer": "Adam lr 1e-2 on per-splat radius scale "
                                                        "(fused, capturable)",
                               "loss_curve": curve, "seconds": fit_s,
                               "graph": "each fit object runs 3 eager steps, captures the step "
                                        "in a CUDA graph and replays it",
                               "checkpoint": "saved after step 100, resumed in a new RadiusFit",
                               "reference_views": target_src,
                               "scale_mean_after": float(scl.detach().mean())},
                       "note": "forward = one LBVH rebuild with the current radius scales + one "
                               "launch tracing all views; backward = one launch of the adjoint "
                               "over all views, accumulated in place; L2 loss vs the reference "
                               "views; forward_backward* are autograd steps (colour, opacity "
                               "and scale gradients), eager and replayed from a CUDA graph "
                               "(*_graphed: GPU time, the eager step's host issue time depends on "
                               "the host); fit_step* is the fit's step (the LBVH refitted to "
                               "the new radius scales, the scale gradient and the Adam update), "
                               "eager and graph-replayed"}

    # ---------------- CPU oracle on the host cores (rank 0, N = 1) ------------------------------
    if rank == 0 and world == 1:
        import oracle
        oracle.build()
        rgba, depth, srv, clis = groups[0]
        cli_objs = W.client_poses()[:FRAMES_PER_IMAGE]
        threads = oracle.default_threads()
        t, r, det = oracle_step_time(rgba.cpu().numpy(), depth.cpu().numpy(), srv, cli_objs,
                                     ray_stride=8, threads=threads)
        line["cpu_baseline"] = {"value": r / t / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": "one step of the large workload: unproject and BVH build "
                                          "over all splats, every 8th ray of the 4 frames traced and "
                                          "the trace time scaled to all rays",
                                "detail": det}
        line["parity"] = parity_budget(wrs, torch, synth, params, leaf)


if __name__ == "__main__":
    main()
