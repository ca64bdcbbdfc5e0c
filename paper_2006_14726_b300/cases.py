"""Run one workload of the hot path once, with few launches, for profiling and inspection.

    python -m paper_2006_14726_b300.cases large --frames 3 [--leaf 1 --k 1 --block 128 --schedule 1]
    python -m paper_2006_14726_b300.cases diff [--leaf 1 --k 4 --schedule 2]
    python -m paper_2006_14726_b300.cases batched --sessions 16 [--k 1 --schedule 0]

Sets up the server image with the GPU ray caster, frees the volume, then runs unproject, the
LBVH build and ``frames`` client traces (each stage in its own NVTX range) and prints the CUDA
event times.  Workloads: tiny, mid, large (see synth).  ``diff``: the differentiable workload
(256^3 blobs, 512^2 server image, 8 views of 512^2, soft edges 0.25): two forward + backward
steps of the 8 views (one launch each way per step) against the ray-cast views.  ``batched``:
the first ``sessions`` of the multi-session workload (server images of 256^2 to 1024^2, 1024^2
clients), two launches of wrs_trace_batched (the second one is the one to profile).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import paper_2006_14726_b300 as wrs  # noqa: E402
import synth  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=["tiny", "mid", "large", "diff", "batched"])
    ap.add_argument("--sessions", type=int, default=16)
    ap.add_argument("--frames", type=int, default=3)
    ap.add_argument("--leaf", type=int, default=1)
    ap.add_argument("--k", type=int, default=1)
    ap.add_argument("--block", type=int, default=128)
    ap.add_argument("--max-hits", type=int, default=0)
    ap.add_argument("--schedule", type=int, default=0, help="0 per pixel, 1 persistent, 2 packet")
    ap.add_argument("--width", type=int, default=4, help="2 binary nodes, 4 four-wide nodes")
    a = ap.parse_args()
    if a.workload == "diff":
        diff_case(a)
        return
    if a.workload == "batched":
        batched_case(a)
        return
    W = {"tiny": synth.TINY, "mid": synth.MID, "large": synth.LARGE}[a.workload]
    dev = torch.device("cuda")
    srv = W.server_cam()
    vol = torch.from_numpy(W.volume()).to(dev)
    tf = torch.from_numpy(synth.tf_ramp()).to(dev)
    rgba, depth = wrs.raycast_volume(vol, tf, srv)
    del vol
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    cams = [wrs.make_camera(c) for c in W.client_poses(max(a.frames, 1))][: a.frames]
    params = wrs.TraceParams(max_hits=a.max_hits, k_chunk=a.k, block=a.block, schedule=a.schedule,
                             width=a.width)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 + a.frames)]
    st = wrs.new_status()
    ev[0].record()
    torch.cuda.nvtx.range_push("unproject")
    sp = wrs.unproject(rgba, depth, srv)
    torch.cuda.nvtx.range_pop()
    ev[1].record()
    torch.cuda.nvtx.range_push("lbvh")
    bvh, srt = wrs.build_lbvh(sp, a.leaf)
    torch.cuda.nvtx.range_pop()
    ev[2].record()
    out = torch.empty(W.client_h, W.client_w, 4, device=dev)
    for f, c in enumerate(cams):
        torch.cuda.nvtx.range_push(f"trace{f}")
        wrs.trace(bvh, srt, c, params, out=out, status=st)
        torch.cuda.nvtx.range_pop()
        ev[3 + f].record()
    torch.cuda.synchronize()
    wrs.check_status(st)
    res = {"workload": a.workload, "splats": sp.count(), "unproject_ms": ev[0].elapsed_time(ev[1]),
           "lbvh_ms": ev[1].elapsed_time(ev[2]),
           "trace_ms": [ev[2 + f].elapsed_time(ev[3 + f]) for f in range(a.frames)],
           "device_bytes_allocated": torch.cuda.memory_allocated()}
    print(json.dumps(res))


def diff_case(a):
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
        loss = ((wrs.render_views(sp, views, col, opa, scl, params, a.leaf) - target) ** 2).mean()
        loss.backward()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    print(json.dumps({"workload": "diff", "splats": n, "views": len(views),
                      "fwd_bwd_ms": ms, "loss": float(loss.detach())}))


def batched_case(a):
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


if __name__ == "__main__":
    main()
