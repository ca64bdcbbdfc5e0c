"""GPU parity of the depth heuristics beyond first hit (§2, §5; readings: spec S2a) through the C
ABI: depths bitwise (every decision binary32 with the oracle's operation order), colours within
the ray caster's tolerance, on f32 and u8 volumes."""
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


@pytest.mark.parametrize("h,param", [(0, 0.1), (1, None), (2, 0.5), (2, 0.9), (3, None)])
def test_tiny_full_image(wrs, h, param):
    W = synth.TINY
    cam = W.server_cam()
    vol = W.volume()
    rgba_r, depth_r = oracle.raycast(vol, synth.tf_ramp(), cam, heuristic=h, param=param)
    rgba, depth = wrs.raycast_volume(_cuda(vol), _cuda(synth.tf_ramp()), cam, heuristic=h, param=param)
    assert np.array_equal(depth.cpu().numpy().view(np.uint32), depth_r.view(np.uint32))
    assert np.abs(rgba.cpu().numpy().astype(np.float64) - rgba_r).max() < 1e-5


@pytest.mark.parametrize("h", [1, 2, 3])
def test_u8_iso_ragged(wrs, h):
    """u8 volume (a quantised blob field), iso-band transfer function, ragged 133 x 97 image."""
    vol = (synth.gaussian_volume(48, 8, 77) * 255).round().astype(np.uint8)
    cam = synth.server_camera(1.6, 35.0, 133, 97)
    tf = synth.tf_iso()
    _, depth_r = oracle.raycast(vol, tf, cam, heuristic=h)
    _, depth = wrs.raycast_volume(_cuda(vol), _cuda(tf), cam, heuristic=h)
    assert np.array_equal(depth.cpu().numpy().view(np.uint32), depth_r.view(np.uint32))
    assert np.isfinite(depth_r).mean() > 0.05


def test_unknown_heuristic_rejected(wrs):
    vol = _cuda(np.zeros((4, 4, 4), np.float32))
    with pytest.raises(wrs.WrsError):
        wrs.raycast_volume(vol, _cuda(synth.tf_ramp()), synth.server_camera(1.4, 30.0, 8, 8),
                           heuristic=4)
