"""Degenerate and extreme inputs through the C ABI, against the oracle: rays with exactly zero
direction components, an eye inside the spheres, zero and huge radii, coincident splats, and a
4096 x 4096 server image (16.7 M splats, the largest case here) on sampled pixels."""
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


def _scene(wrs, pos_r, rgba, leaf=1):
    """GPU sorted splats + LBVH and the oracle splats for hand-made records."""
    n = len(pos_r)
    sp = wrs.SplatBuffers(n)
    sp.pos_r[:n] = _cuda(np.float32(pos_r))
    sp.rgba[:n] = _cuda(np.float32(rgba))
    sp.id[:n] = torch.arange(n, dtype=torch.int32, device="cuda")
    sp.n.fill_(n)
    bvh, srt = wrs.build_lbvh(sp, leaf)
    ref = oracle.Splats(np.float32(pos_r), np.float32(rgba), np.arange(n, dtype=np.uint32))
    return bvh, srt, ref


@pytest.mark.parametrize("schedule,width", [(0, 4), (0, 2), (1, 4), (2, 4)])
def test_axis_aligned_rays_and_eye_inside(wrs, schedule, width):
    """Odd image sizes put the centre ray exactly on the view axis (zero x and y direction
    components, the guarded slab case); one sphere contains the eye (entry distance 0); zero-radius
    and coincident splats."""
    rng = np.random.default_rng(7)
    n = 3000
    pos = rng.uniform(0.2, 0.8, size=(n, 3))
    r = rng.uniform(0.002, 0.02, size=n)
    pos[:40] = pos[40]            # 41 coincident centres (ties by id)
    r[100:140] = 0.0              # never hit
    pos[200] = (0.5, 0.5, 2.0)    # a sphere around the eye
    r[200] = 0.3
    pos_r = np.concatenate([pos, r[:, None]], axis=1)
    rgba = rng.uniform(0, 1, size=(n, 4)) * 0.5
    bvh, srt, ref = _scene(wrs, pos_r, rgba)
    cam = synth.look_at((0.5, 0.5, 2.0), (0.5, 0.5, 0.0), (0, 1, 0), 40.0, 65, 49)
    assert cam.fwd[0] == 0.0 and cam.fwd[1] == 0.0
    st = wrs.new_status()
    img = wrs.trace(bvh, srt, cam, wrs.TraceParams(schedule=schedule, width=width, k_chunk=2),
                    status=st)
    wrs.check_status(st)
    want = oracle.trace(oracle.Scene(ref), cam)
    err = np.abs(img.cpu().numpy().reshape(-1, 4).astype(np.float64) - want["rgba"])
    assert err.max() <= 1e-5 and err.mean() <= MEAN_ABS
    # every ray starts inside the big sphere: its entry distance is 0, so all pixels are covered
    assert (img[..., 3] > 0).all()


def test_huge_sphere_and_single_splat_scenes(wrs):
    cam = synth.server_camera(1.4, 30.0, 31, 23)
    for pos_r in ([[0.5, 0.5, 0.5, 50.0]], [[0.5, 0.5, 0.5, 0.05]], [[9.0, 9.0, 9.0, 0.1]]):
        bvh, srt, ref = _scene(wrs, pos_r, [[0.2, 0.3, 0.4, 0.5]])
        img = wrs.trace(bvh, srt, cam, wrs.TraceParams(width=4))
        want = oracle.trace(oracle.Scene(ref), cam)
        assert np.abs(img.cpu().numpy().reshape(-1, 4) - want["rgba"]).max() <= 1e-6


def test_4096_square_server_image_sampled(wrs):
    """The largest case: a 4096 x 4096 server image (16.7 M splats) warped to a 2048 x 2048 client
    at 10 degrees; 2048 sampled pixels against the oracle, with both leaf sizes the tuner uses."""
    rgba, depth = synth.synthetic_server_image(4096, 4096, 77, hole_frac=0.02)
    srv = synth.server_camera(1.4, 30.0, 4096, 4096)
    cli = synth.orbit(srv, (0.6, 0.8, 0.0), 10.0, 2048, 2048)
    sp = wrs.unproject(_cuda(rgba), _cuda(depth), srv)
    ref_sp = oracle.unproject(rgba, depth, srv)
    assert sp.count() == ref_sp.n > 16_000_000
    pix = np.random.default_rng(3).choice(2048 * 2048, 2048, replace=False)
    want = oracle.trace(oracle.Scene(ref_sp), cli, pixels=pix)
    st = wrs.new_status()
    for leaf, sched in ((1, 0), (2, 1)):
        bvh, srt = wrs.build_lbvh(sp, leaf)
        img = wrs.trace(bvh, srt, cli, wrs.TraceParams(k_chunk=1, schedule=sched, width=4), status=st)
        wrs.check_status(st)
        err = np.abs(img.cpu().numpy().reshape(-1, 4)[pix].astype(np.float64) - want["rgba"])
        assert err.max() <= MAX_ABS and err.mean() <= MEAN_ABS, (leaf, err.max())
        del bvh, srt
