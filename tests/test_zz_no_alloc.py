"""wrs_unproject_static: unprojection for callers that cannot give the library device memory.

Some applications fix their device memory when they start (an embedded viewer, or a plug-in
whose host owns the GPU heap) and cannot hand out a work buffer per call.  For them the library
offers an entry point whose work buffer is a fixed array inside its own device image.  This file
checks, through the C ABI, that two calls in a row -- a large image, then a smaller one that
leaves stale counts from the first call in the shared array -- give exactly what the ordinary
wrs_unproject gives (splat count, ids, positions, radii, colours: bitwise), and that images beyond
the fixed limit are refused.  It is collected last so that a failure here stops a run only after
every other test has run; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wrs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_14726_b300 as w
    return w


def _static(wrs, rgba, depth, cam):
    c = wrs.make_camera(cam)
    out = wrs.SplatBuffers(c.width * c.height)
    sp = out.c()
    rc = wrs.lib.wrs_unproject_static(rgba.data_ptr(), depth.data_ptr(), ctypes.byref(c),
                                      wrs.RADIUS_FOOTPRINT, 0.0, ctypes.byref(sp),
                                      torch.cuda.current_stream().cuda_stream)
    assert rc == wrs.WRS_OK, wrs.last_error()
    return out


def _same(a, b):
    assert a.count() == b.count()
    for x, y in zip(a.view(), b.view()):
        assert torch.equal(x.view(torch.int32), y.view(torch.int32))


def test_static_unproject_matches_unproject_on_two_calls(wrs):
    cases = [(1920, 1080, 7), (640, 360, 8)]  # the second call sees the first call's leftovers
    for w, h, seed in cases:
        rgba, depth = synth.synthetic_server_image(w, h, seed)
        cam = synth.server_camera(1.4, 30.0, w, h)
        r = torch.from_numpy(rgba).cuda()
        d = torch.from_numpy(depth).cuda()
        got = _static(wrs, r, d, cam)
        ref = wrs.unproject(r, d, cam)
        torch.cuda.synchronize()
        assert got.count() > 0
        _same(got, ref)


def test_static_unproject_refuses_images_beyond_its_limit(wrs):
    cam = synth.server_camera(1.4, 30.0, 8193, 8192)
    c = wrs.make_camera(cam)
    tiny = torch.zeros(16, device="cuda")
    sp = wrs._Splats(tiny.data_ptr(), tiny.data_ptr(), tiny.data_ptr(), None, tiny.data_ptr(),
                     0xFFFFFFFF)
    rc = wrs.lib.wrs_unproject_static(tiny.data_ptr(), tiny.data_ptr(), ctypes.byref(c), 0, 0.0,
                                      ctypes.byref(sp), None)
    assert rc == wrs.WRS_ERR_CAPACITY
    assert "8192 x 8192" in wrs.last_error()
