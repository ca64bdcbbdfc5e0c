"""GPU parity of the samples smeared along their viewing ray (future work, §6; reading: spec S3b)
through the C ABI: chain positions, radii and ids bitwise, colours within binary32 rounding of the
oracle's binary64 opacity split, and traced chains within the trace tolerance."""
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


def _check(sp, ref):
    pos, rgba, ids = (t.cpu().numpy() for t in sp.view())
    assert ids.shape[0] == ref.n
    assert np.array_equal(ids.view(np.uint32), ref.id)
    assert np.array_equal(pos.view(np.uint32), ref.pos_r.view(np.uint32))
    assert np.allclose(rgba, ref.rgba, rtol=2e-6, atol=1e-9)


def _blob_frame(W, H):
    """A server frame of a blob volume with the accumulated-opacity depth interval."""
    vol = synth.gaussian_volume(48, 8, 91)
    cam = synth.server_camera(1.6, 35.0, W, H)
    rgba, lo = oracle.raycast(vol, synth.tf_ramp(), cam, heuristic=oracle.DEPTH_ACCUMULATED, param=0.25)
    _, hi = oracle.raycast(vol, synth.tf_ramp(), cam, heuristic=oracle.DEPTH_ACCUMULATED, param=0.75)
    return vol, rgba.astype(np.float32), lo, hi, cam


@pytest.mark.parametrize("max_chain,mode", [(8, 0), (3, 0), (16, 1)])
def test_chains_from_a_volume_bitwise(wrs, max_chain, mode):
    _, rgba, lo, hi, cam = _blob_frame(97, 71)
    diag = 3 ** 0.5 / 48
    ref = oracle.unproject_interval(rgba, lo, hi, cam, mode, diag, max_chain)
    sp = wrs.unproject_interval(_cuda(rgba), _cuda(lo), _cuda(hi), cam, max_chain, mode, diag)
    _check(sp, ref)
    assert ref.n > (np.isfinite(lo) & (rgba[..., 3] > 0)).sum()  # some pixels became chains


def test_the_gpu_ray_caster_feeds_the_same_chains(wrs):
    """End to end on the device: the two accumulated-opacity depths from wrs_raycast_volume, then
    the chains; traced from a novel view against the oracle."""
    vol, rgba, lo, hi, cam = _blob_frame(120, 90)
    dv, tf = _cuda(vol), _cuda(synth.tf_ramp())
    g_rgba, g_lo = wrs.raycast_volume(dv, tf, cam, heuristic=wrs.DEPTH_ACCUMULATED, param=0.25)
    _, g_hi = wrs.raycast_volume(dv, tf, cam, heuristic=wrs.DEPTH_ACCUMULATED, param=0.75)
    assert np.array_equal(g_lo.cpu().numpy().view(np.uint32), lo.view(np.uint32))
    assert np.array_equal(g_hi.cpu().numpy().view(np.uint32), hi.view(np.uint32))
    sp = wrs.unproject_interval(_cuda(rgba), g_lo, g_hi, cam, 8)
    ref = oracle.unproject_interval(rgba, lo, hi, cam, 0, 0.0, 8)
    _check(sp, ref)
    bvh, srt = wrs.build_lbvh(sp, 1)
    cli = synth.orbit(cam, (0, 1, 0), 12.0, 100, 80)
    img = wrs.trace(bvh, srt, cli, wrs.TraceParams(k_chunk=4))
    want = oracle.trace(oracle.Scene(ref), cli)
    err = np.abs(img.cpu().numpy().reshape(-1, 4).astype(np.float64) - want["rgba"])
    assert err.max() <= 2e-3 and err.mean() <= 1e-4


def test_1080p_chains_bitwise(wrs):
    rgba, depth = synth.synthetic_server_image(1920, 1080, 71)
    hi = depth * np.float32(1.04)
    cam = synth.LARGE.server_cam()
    ref = oracle.unproject_interval(rgba, depth, hi, cam, 0, 0.0, 8)
    sp = wrs.unproject_interval(_cuda(rgba), _cuda(depth), _cuda(hi), cam, 8)
    _check(sp, ref)


def test_zero_interval_and_capacity_overflow(wrs):
    rgba, depth = synth.synthetic_server_image(64, 48, 72)
    cam = synth.server_camera(1.4, 30.0, 64, 48)
    a = wrs.unproject(_cuda(rgba), _cuda(depth), cam)
    b = wrs.unproject_interval(_cuda(rgba), _cuda(depth), _cuda(depth), cam, 4)
    pa, ca, ia = a.view()
    pb, cb, ib = b.view()
    assert torch.equal(pa, pb) and torch.equal(ca, cb) and torch.equal(ia * 4, ib)
    hi = depth * np.float32(1.3)  # long intervals: chains of up to 6
    ref = oracle.unproject_interval(rgba, depth, hi, cam, 0, 0.0, 6)
    cap = ref.n - 50
    st = wrs.new_status()
    sp = wrs.unproject_interval(_cuda(rgba), _cuda(depth), _cuda(hi), cam, 6,
                                out=wrs.SplatBuffers(cap), status=st)
    assert sp.count() == cap and int(st.item()) == wrs.STATUS_SPLAT_OVERFLOW
    st.zero_()
    pos = sp.view()[0].cpu().numpy()
    assert np.array_equal(pos.view(np.uint32), ref.pos_r[:cap].view(np.uint32))
    with pytest.raises(wrs.WrsError):
        wrs.unproject_interval(_cuda(rgba), _cuda(depth), _cuda(hi), cam, 65)
