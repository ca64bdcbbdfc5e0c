"""GPU parity of the point-splat warping (the earlier method the paper compares against, §2, §5,
Fig. 3; reading: spec S10) through the C ABI: the index of the point each pixel shows and its
colour must match the oracle bitwise (every decision is binary32 with the same operation order).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wrs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_14726_b300 as w
    oracle.build()
    return w


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check(wrs, rgba, depth, srv, cli, size):
    ref_sp = oracle.unproject(rgba, depth, srv)
    sp = wrs.unproject(_cuda(rgba), _cuda(depth), srv)
    idx = torch.empty(cli.height, cli.width, dtype=torch.int32, device="cuda")
    img = wrs.point_splat(sp, cli, size, index=idx)
    ref_img, ref_idx = oracle.point_splat(ref_sp, cli, size)
    assert np.array_equal(idx.cpu().numpy().astype(np.int64), ref_idx)
    assert np.array_equal(img.cpu().numpy().view(np.uint32), ref_img.view(np.uint32))
    return ref_idx


@pytest.mark.parametrize("size", [1, 2, 3, 5])
def test_tiny_full_image_bitwise(wrs, size):
    W = synth.TINY
    srv = W.server_cam()
    rgba, depth = oracle.raycast(W.volume(), synth.tf_ramp(), srv)
    idx = _check(wrs, rgba.astype(np.float32), depth, srv, synth.tiny_client_camera(), size)
    assert (idx >= 0).mean() > 0.2


def test_ragged_client_and_identity_view(wrs):
    rgba, depth = synth.synthetic_server_image(133, 97, 12)
    srv = synth.server_camera(1.4, 30.0, 133, 97)
    _check(wrs, rgba, depth, srv, srv, 1)
    _check(wrs, rgba, depth, srv, synth.orbit(srv, (0, 1, 0), 25.0, 101, 77), 4)


@pytest.mark.parametrize("size", [1, 3])
def test_1080p_full_image_bitwise(wrs, size):
    """Full size: 1920 x 1080 server image (about 2 M points) warped to a 1920 x 1080 client 20
    degrees away; every pixel compared."""
    rgba, depth = synth.synthetic_server_image(1920, 1080, 51)
    srv = synth.LARGE.server_cam()
    _check(wrs, rgba, depth, srv, synth.orbit(srv, (0.6, 0.8, 0.0), 20.0), size)


def test_empty_set_and_eye_inside_the_cloud(wrs):
    srv = synth.server_camera(1.4, 30.0, 16, 8)
    sp = wrs.SplatBuffers(16 * 8)
    img = wrs.point_splat(sp, srv, 3)
    assert not img.any()
    # a client eye in the middle of the cloud: points behind it are dropped
    rgba, depth = synth.synthetic_server_image(64, 48, 13)
    srv = synth.server_camera(1.4, 30.0, 64, 48)
    cli = synth.look_at((0.5, 0.5, 0.5), (0.5, 0.5, 2.0), (0, 1, 0), 60.0, 64, 48)
    _check(wrs, rgba, depth, srv, cli, 2)


def test_rejects_bad_arguments(wrs):
    srv = synth.server_camera(1.4, 30.0, 16, 8)
    sp = wrs.SplatBuffers(16 * 8)
    for s in (0, 65):
        with pytest.raises(wrs.WrsError):
            wrs.point_splat(sp, srv, s)
    with pytest.raises(wrs.WrsError):
        wrs.point_splat(sp, srv, 1, scratch=torch.empty(8, dtype=torch.uint8, device="cuda"))


def test_quality_table_identity_pose_is_exact(wrs):
    """At the server's own pose the 1-pixel point warp reproduces the server image, which is the
    ray caster's image at that pose: PSNR = inf; other poses give finite scores."""
    from paper_2006_14726_b300.quality import warp_quality
    vol = synth.gaussian_volume_device(64, 16, 77)
    tf = torch.from_numpy(synth.tf_ramp()).cuda()
    srv = synth.server_camera(1.4, 30.0, 160, 120)
    rows = warp_quality(vol, tf, srv, [srv, synth.orbit(srv, (0, 1, 0), 8.0)])
    assert rows[0]["points_1px"] == float("inf") and rows[0]["server_view_unwarped"] == float("inf")
    for k, v in rows[1].items():
        assert v is not None and 5.0 < v < 200.0, (k, v)
