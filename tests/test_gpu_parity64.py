"""GPU trace against the binary64-decision oracle (Fig. 2 caption, §4), through the C ABI.

The tolerance clause of the parity budget: per-pixel RGBA max abs <= 2e-3 and mean abs <= 1e-4
against an oracle whose every decision (primary ray, hit or miss, entry distance, hit order) is
binary64, excluding only tie pixels -- a move of the ray or a sphere by at most 1e-6 can change
which spheres they composite or their order -- and at most 0.1 % of the pixels.  The excluded
pixels are the ones beyond the tolerance; each must be a tie, and they are listed (printed).

Cases: the tiny workload (full image; first hit, all hits, soft edge), the mid workload (1024^2
client over the 512^2 ray-cast server image, full image) and three poses of the large
workload's cap on the 1080p stand-in server image (about 2 M splats, full images) in the
launch the benchmark times and in the other schedules.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_ABS = 2e-3
MEAN_ABS = 1e-4
BUDGET = 1e-3


@pytest.fixture(scope="module")
def wrs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_14726_b300 as w
    oracle.build()
    return w


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check_budget(gpu, ref, what):
    """Exclusions = pixels beyond the tolerance; all must be ties, at most 0.1 % of the image."""
    gpu = np.asarray(gpu, np.float64).reshape(-1, 4)
    err = np.abs(gpu - ref["rgba"])
    worst = err.max(1)
    excluded = worst > MAX_ABS
    npix = worst.size
    listed = np.flatnonzero(excluded)
    not_tie = np.flatnonzero(excluded & ~ref["tie"])
    print(f"{what}: {npix} px, ties {int(ref['tie'].sum())}, excluded {listed.size} "
          f"({listed.size / max(npix, 1):.4%}): {listed[:20].tolist()}{' ...' if listed.size > 20 else ''}")
    assert not_tie.size == 0, f"{what}: pixels beyond tolerance that are not ties: {not_tie[:10]}"
    assert listed.size <= BUDGET * npix, f"{what}: {listed.size} excluded pixels"
    rest = err[~excluded]
    if rest.size:
        assert rest.max() <= MAX_ABS, f"{what}: max abs {rest.max():.3g}"
        assert rest.mean() <= MEAN_ABS, f"{what}: mean abs {rest.mean():.3g}"
    return listed


def _gpu_scene(wrs, rgba, depth, srv, leaf=1):
    sp = wrs.unproject(_cuda(rgba), _cuda(depth), srv)
    return wrs.build_lbvh(sp, leaf)


@pytest.mark.parametrize("H,beta", [(0, 0.0), (1, 0.0), (0, 0.25)])
def test_tiny_full_image_vs_binary64(wrs, H, beta):
    W = synth.TINY
    srv = W.server_cam()
    rgba, depth = oracle.raycast(W.volume(), synth.tf_ramp(), srv)
    rgba = rgba.astype(np.float32)
    cli = synth.tiny_client_camera()
    bvh, srt = _gpu_scene(wrs, rgba, depth, srv)
    img = wrs.trace(bvh, srt, cli, wrs.TraceParams(max_hits=H, edge_softness=beta))
    ref = oracle.trace64(oracle.Scene(oracle.unproject(rgba, depth, srv), max_hits=H, beta=beta), cli)
    check_budget(img.cpu().numpy(), ref, f"tiny H={H} beta={beta}")


def test_mid_full_image_vs_binary64(wrs):
    W = synth.MID
    srv = W.server_cam()
    rgba, depth = oracle.raycast(W.volume(), synth.tf_ramp(), srv)
    rgba = rgba.astype(np.float32)
    cli = W.client_poses(3)[2]
    bvh, srt = _gpu_scene(wrs, rgba, depth, srv)
    img = wrs.trace(bvh, srt, cli, wrs.TraceParams(k_chunk=1, schedule=wrs.SCHEDULE_PACKET, width=4))
    ref = oracle.trace64(oracle.Scene(oracle.unproject(rgba, depth, srv)), cli)
    check_budget(img.cpu().numpy(), ref, "mid 1024^2")


@pytest.fixture(scope="module")
def large(wrs):
    rgba, depth = synth.synthetic_server_image(1920, 1080, 52)
    srv = synth.LARGE.server_cam()
    bvh, srt = _gpu_scene(wrs, rgba, depth, srv)
    scene = oracle.Scene(oracle.unproject(rgba, depth, srv))
    return bvh, srt, scene, oracle.BVH(scene)


@pytest.mark.parametrize("pose", [5, 23, 41])
def test_large_full_images_vs_binary64(wrs, large, pose):
    """The benchmark's launch (one thread per pixel, 4-wide nodes, K 1, leaf 1) on full 1080p
    images, and the persistent and packet schedules on the same frames."""
    bvh, srt, scene, obvh = large
    cli = synth.LARGE.client_poses()[pose]
    ref = oracle.trace64(scene, cli, bvh=obvh)
    for sched, k in ((wrs.SCHEDULE_PER_PIXEL, 1), (wrs.SCHEDULE_PERSISTENT, 2), (wrs.SCHEDULE_PACKET, 4)):
        img = wrs.trace(bvh, srt, cli, wrs.TraceParams(k_chunk=k, schedule=sched, width=4))
        check_budget(img.cpu().numpy(), ref, f"large pose {pose} schedule {sched}")
