"""The batched multi-session trace against the oracle at the batched workload's shape.

One session per server size of the batched workload (256^2, 384^2, 512^2, 768^2, 1024^2), each
with its own seeded 256^3 blob volume ray-cast by the oracle, its own camera offset within 15
degrees and a 1024^2 client, all traced in one launch under every schedule (one warp per tile,
persistent, warp-shared traversal per tile, and each session's own schedule as the tuner picks
it).  4096 sampled pixels per session against the binary32-decision oracle (identical hit lists:
compositing rounding only) and against the binary64-decision oracle within the tie budget.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_ABS = 2e-3
MEAN_ABS = 1e-4


@pytest.fixture(scope="module")
def wrs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_14726_b300 as w
    oracle.build()
    return w


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def sessions(wrs):
    tf = synth.tf_ramp()
    out = []
    for s, size in enumerate(synth.BATCHED_SERVER_SIZES):
        srv = synth.BATCHED.server_cam(size, size)
        rgba, depth = oracle.raycast(synth.BATCHED.volume(seed_offset=s), tf, srv)
        rgba = rgba.astype(np.float32)
        cli = synth.poses_in_cap(srv, 1, synth.BATCHED.cap_deg, 4100 + s, synth.BATCHED.client_w,
                                 synth.BATCHED.client_h)[0]
        sp = wrs.unproject(_cuda(rgba), _cuda(depth), srv)
        bvh, srt = wrs.build_lbvh(sp, 1)
        ref_sp = oracle.unproject(rgba, depth, srv)
        assert sp.count() == ref_sp.n
        scene = oracle.Scene(ref_sp)
        pix = np.random.default_rng(200 + s).choice(cli.width * cli.height, 4096, replace=False)
        obvh = oracle.BVH(scene)
        out.append({"gpu": (bvh, srt, cli), "pix": pix,
                    "ref": oracle.trace(scene, cli, pixels=pix, bvh=obvh),
                    "ref64": oracle.trace64(scene, cli, pixels=pix, bvh=obvh)})
    return out


@pytest.mark.parametrize("sched,k,width", [(0, 1, 4), (0, 4, 2), (1, 2, 4), (2, 4, 4), (2, 1, 2),
                                           (3, 1, 4), (3, 4, 4)])
def test_batched_sessions_against_oracle(wrs, sessions, sched, k, width):
    batch = wrs.Batch([s["gpu"] for s in sessions])
    if sched == wrs.SCHEDULE_PER_SESSION:
        # the tuner's mix: warp-shared traversal for the sparse sessions, per pixel for the rest
        assert set(batch.schedules) == {wrs.SCHEDULE_PACKET, wrs.SCHEDULE_PER_PIXEL}
    for o in batch.outputs:
        o.fill_(-1.0)
    st = wrs.new_status()
    outs = wrs.trace_batched(batch, wrs.TraceParams(k_chunk=k, width=width, schedule=sched),
                             status=st)
    wrs.check_status(st)
    for s, (o, ses) in enumerate(zip(outs, sessions)):
        got = o.cpu().numpy().reshape(-1, 4)[ses["pix"]].astype(np.float64)
        err = np.abs(got - ses["ref"]["rgba"])
        what = f"session {s} ({synth.BATCHED_SERVER_SIZES[s]}^2 server) schedule {sched} K {k}"
        assert err.max() <= 1e-5, f"{what}: max abs {err.max():.3g}"  # identical hit lists
        assert err.mean() <= MEAN_ABS, what
        # binary64 decisions: only ties beyond the tolerance, at most 0.1 % of the samples
        err64 = np.abs(got - ses["ref64"]["rgba"]).max(1)
        excl = err64 > MAX_ABS
        assert not np.any(excl & ~ses["ref64"]["tie"]), what
        assert np.count_nonzero(excl) <= 1e-3 * excl.size + 1, what
        assert err64[~excl].mean() <= MEAN_ABS, what


def test_batched_one_launch_equals_sessions_traced_alone(wrs, sessions):
    """The same sessions: one launch of the tuner's per-session mix equals each session traced
    alone with its own schedule, bitwise."""
    batch = wrs.Batch([s["gpu"] for s in sessions])
    outs = wrs.trace_batched(batch, wrs.TraceParams(k_chunk=1, width=4,
                                                    schedule=wrs.SCHEDULE_PER_SESSION))
    for (bvh, srt, cli), sched, o in zip([s["gpu"] for s in sessions], batch.schedules, outs):
        alone = wrs.trace(bvh, srt, cli, wrs.TraceParams(k_chunk=1, width=4, schedule=sched))
        assert torch.equal(o.view(torch.int32), alone.view(torch.int32))
