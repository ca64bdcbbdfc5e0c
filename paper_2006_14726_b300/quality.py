"""Image quality of the warped views, the paper's Fig. 3 comparison restated as numbers.

Fig. 3 shows, for a sequence of client poses moving away from the server's, the view warped from
one server image by (a) ray-traced sphere splats and (b) the earlier point rasterisation, next to
the volume rendered directly at each pose.  Here each warped view is scored by its PSNR against the
server ray caster run at the client pose (spec S10): all images come from this library's kernels
(wrs_raycast_volume, wrs_unproject, wrs_build_lbvh, wrs_trace, wrs_point_splat); the PSNR itself is
evaluation, computed with torch.
"""
from __future__ import annotations

import math
from typing import Dict, Iterable, List

import torch

from . import (DEPTH_ACCUMULATED, RADIUS_VOXEL, TraceParams, build_lbvh, make_camera, point_splat,
               raycast_volume, trace, unproject, unproject_interval)


def psnr(img: torch.Tensor, ref: torch.Tensor) -> float:
    """10 log10(1 / MSE) over all channels (images in [0, 1])."""
    mse = float(torch.mean((img.double() - ref.double()) ** 2))
    return math.inf if mse == 0.0 else 10.0 * math.log10(1.0 / mse)


def warp_quality(vol: torch.Tensor, tf: torch.Tensor, srv, clients: Iterable,
                 point_sizes: Iterable[int] = (1, 2, 3), max_hits: Iterable[int] = (0, 1),
                 sphere_scales: Iterable[float] = (1.0, 2.0), voxel_diag: float = 0.0,
                 step_vox: float = 0.5, tau: float = 0.1, leaf_size: int = 1,
                 heuristic: int = 0, heuristic_param=None, interval_chain: int = 0) -> List[Dict]:
    """PSNR of every warping method for each client pose; one dict per pose.

    Sphere variants: the footprint radius scaled by each of ``sphere_scales`` (composited with
    each of ``max_hits``; 1 = the paper's first-hit query), and, if ``voxel_diag`` > 0, the
    paper's own radius rule (half a voxel diagonal, §4.1) with first hit.  Point variants: each
    of ``point_sizes`` pixels.  ``heuristic`` picks the server's depth rule (DEPTH_*); the
    ground truth's colours do not depend on it.  ``interval_chain`` > 0 adds samples smeared along
    their rays over the depth interval of growing opacity (chains of up to that many spheres)."""
    rgba, depth = raycast_volume(vol, tf, srv, step_vox, tau, heuristic=heuristic,
                                 param=heuristic_param)
    sp = unproject(rgba, depth, srv)
    trees = {f"spheres_x{g:g}": build_lbvh(sp, leaf_size, global_scale=g) for g in sphere_scales}
    if voxel_diag > 0.0:
        spv = unproject(rgba, depth, srv, RADIUS_VOXEL, voxel_diag)
        trees["spheres_voxel"] = build_lbvh(spv, leaf_size)
    if interval_chain > 0:
        _, d_lo = raycast_volume(vol, tf, srv, step_vox, heuristic=DEPTH_ACCUMULATED, param=0.25)
        _, d_hi = raycast_volume(vol, tf, srv, step_vox, heuristic=DEPTH_ACCUMULATED, param=0.75)
        spi = unproject_interval(rgba, d_lo, d_hi, srv, interval_chain)
        trees["spheres_interval"] = build_lbvh(spi, leaf_size)
    rows = []
    for cli in clients:
        c = make_camera(cli)
        truth, _ = raycast_volume(vol, tf, c, step_vox, tau)
        row = {}
        for name, (bvh, srt) in trees.items():
            for h in ((1,) if name == "spheres_voxel" else (0,) if name == "spheres_interval"
                      else max_hits):
                img = trace(bvh, srt, c, TraceParams(max_hits=h, width=4))
                row[f"{name}_H{h}"] = psnr(img, truth)
        for s in point_sizes:
            row[f"points_{s}px"] = psnr(point_splat(sp, c, s), truth)
        same = (c.width, c.height) == (srv.width, srv.height)
        row["server_view_unwarped"] = psnr(rgba, truth) if same else None
        rows.append(row)
    return rows
