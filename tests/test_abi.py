"""The C ABI library loads on a machine without a GPU, exports every entry point that
include/wrs.h declares, and rejects bad arguments on the host before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wrs.h")


@pytest.fixture(scope="module")
def wrs():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "wrs_build", os.path.join(ROOT, "paper_2006_14726_b300", "_build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.build()  # rebuilds only if a source is newer than the library
    import paper_2006_14726_b300 as w
    return w


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wrs_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("wrs_unproject", "wrs_build_lbvh", "wrs_trace", "wrs_trace_batched",
                     "wrs_trace_backward", "wrs_raycast_volume"):
        assert required in names


def test_every_declared_symbol_is_exported(wrs):
    lib = ctypes.CDLL(wrs.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match(wrs):
    assert wrs.lib.wrs_camera_size() == ctypes.sizeof(wrs.Camera) == 60
    assert wrs.lib.wrs_session_size() == ctypes.sizeof(wrs.Session)


def test_size_queries(wrs):
    assert wrs.unproject_scratch_bytes(1920, 1080) >= 2 * 4 * ((1920 * 1080 + 1023) // 1024)
    assert wrs.unproject_scratch_bytes(0, 5) == 0
    assert wrs.lib.wrs_lbvh_bytes(1000, 1) == 64 + (64 + 128) * 999
    assert wrs.lib.wrs_lbvh_bytes(1000, 4) == 64 + (64 + 128) * 249
    assert wrs.lib.wrs_lbvh_bytes(10, 0) == 0 and wrs.lib.wrs_lbvh_bytes(10, 17) == 0
    assert wrs.lbvh_scratch_bytes(2_073_600, 1) > 4 * 4 * 2_073_600
    assert wrs.session_tiles(1024, 1024) == 128 * 256 and wrs.session_tiles(17, 1) == 3


def _cam(wrs, w=8, h=8, **kw):
    c = wrs.Camera()
    c.eye[:] = [0.5, 0.5, 2.0]
    c.right[:] = [1, 0, 0]
    c.up[:] = [0, 1, 0]
    c.fwd[:] = [0, 0, -1]
    c.tan_half_fovy = 0.4
    c.width, c.height = w, h
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def test_host_validation_without_device(wrs):
    """Argument errors are reported before any CUDA call (these run with no GPU present)."""
    lib = wrs.lib
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: validation fails first
    sp = wrs._Splats(fake.value, fake.value, fake.value, None, fake.value, 10)
    # NULL image
    assert lib.wrs_unproject(None, fake, ctypes.byref(_cam(wrs)), 0, 0.0, ctypes.byref(sp), fake, 1 << 20, None) == wrs.WRS_ERR_ARG
    assert "NULL" in wrs.last_error()
    # capacity below the pixel count
    assert lib.wrs_unproject(fake, fake, ctypes.byref(_cam(wrs)), 0, 0.0, ctypes.byref(sp), fake, 1 << 20, None) == wrs.WRS_ERR_CAPACITY
    # bad camera
    assert lib.wrs_unproject(fake, fake, ctypes.byref(_cam(wrs, w=0)), 0, 0.0, ctypes.byref(sp), fake, 1 << 20, None) == wrs.WRS_ERR_ARG
    bad = _cam(wrs)
    bad.tan_half_fovy = float("nan")
    assert lib.wrs_unproject(fake, fake, ctypes.byref(bad), 0, 0.0, ctypes.byref(sp), fake, 1 << 20, None) == wrs.WRS_ERR_ARG
    # unknown radius mode, voxel mode without a voxel size
    big = wrs._Splats(fake.value, fake.value, fake.value, None, fake.value, 64)
    assert lib.wrs_unproject(fake, fake, ctypes.byref(_cam(wrs)), 7, 0.0, ctypes.byref(big), fake, 1 << 20, None) == wrs.WRS_ERR_ARG
    assert lib.wrs_unproject(fake, fake, ctypes.byref(_cam(wrs)), 1, 0.0, ctypes.byref(big), fake, 1 << 20, None) == wrs.WRS_ERR_ARG
    # scratch too small
    assert lib.wrs_unproject(fake, fake, ctypes.byref(_cam(wrs)), 0, 0.0, ctypes.byref(big), fake, 1, None) == wrs.WRS_ERR_SCRATCH
    # append: weight outside (0, 1], ids past 2^32, zero capacity (any other capacity is legal)
    args = (fake, fake, ctypes.byref(_cam(wrs)), 0, 0.0)
    assert lib.wrs_unproject_append(*args, 0.0, 0, ctypes.byref(sp), fake, 1 << 20, None, None) == wrs.WRS_ERR_ARG
    assert lib.wrs_unproject_append(*args, 1.5, 0, ctypes.byref(sp), fake, 1 << 20, None, None) == wrs.WRS_ERR_ARG
    assert lib.wrs_unproject_append(*args, 1.0, 2**32 - 63, ctypes.byref(sp), fake, 1 << 20, None, None) == wrs.WRS_ERR_ARG
    assert "2^32" in wrs.last_error()
    zero = wrs._Splats(fake.value, fake.value, fake.value, None, fake.value, 0)
    assert lib.wrs_unproject_append(*args, 1.0, 0, ctypes.byref(zero), fake, 1 << 20, None, None) == wrs.WRS_ERR_CAPACITY
    assert lib.wrs_unproject_append(*args, 1.0, 0, ctypes.byref(sp), fake, 1, None, None) == wrs.WRS_ERR_SCRATCH
    # codec: empty box axis, non-positive radius bound, capacity below the pixel count
    good = wrs.make_codec((0, 0, 0), (1, 1, 1), 0.01)
    flat = wrs.make_codec((0, 0, 0), (1, 1, 0), 0.01)
    norad = wrs.make_codec((0, 0, 0), (1, 1, 1), 0.0)
    for cd in (flat, norad):
        assert lib.wrs_unproject_encode(fake, fake, ctypes.byref(_cam(wrs)), 0, 0.0, ctypes.byref(cd), fake, fake, fake, 64, fake, 1 << 20, None) == wrs.WRS_ERR_ARG
    assert "codec" in wrs.last_error()
    assert lib.wrs_unproject_encode(fake, fake, ctypes.byref(_cam(wrs)), 0, 0.0, ctypes.byref(good), fake, fake, fake, 10, fake, 1 << 20, None) == wrs.WRS_ERR_CAPACITY
    assert lib.wrs_encode_splats(ctypes.byref(big), ctypes.byref(flat), fake, fake, None, None) == wrs.WRS_ERR_ARG
    assert lib.wrs_decode_splats(fake, fake, fake, 65, ctypes.byref(good), ctypes.byref(big), None) == wrs.WRS_ERR_CAPACITY
    # LBVH: bad leaf size, missing src, small capacity
    bv = wrs._Lbvh(fake.value, 64, 0)
    srt = wrs._Splats(fake.value, fake.value, fake.value, fake.value, fake.value, 64)
    assert lib.wrs_build_lbvh(ctypes.byref(big), None, 1.0, ctypes.byref(bv), ctypes.byref(srt), fake, 1 << 30, None) == wrs.WRS_ERR_ARG
    nosrc = wrs._Splats(fake.value, fake.value, fake.value, None, fake.value, 64)
    bv1 = wrs._Lbvh(fake.value, 64, 1)
    assert lib.wrs_build_lbvh(ctypes.byref(big), None, 1.0, ctypes.byref(bv1), ctypes.byref(nosrc), fake, 1 << 30, None) == wrs.WRS_ERR_ARG
    small = wrs._Lbvh(fake.value, 8, 1)
    assert lib.wrs_build_lbvh(ctypes.byref(big), None, 1.0, ctypes.byref(small), ctypes.byref(srt), fake, 1 << 30, None) == wrs.WRS_ERR_CAPACITY
    assert lib.wrs_build_lbvh(ctypes.byref(big), None, 1.0, ctypes.byref(bv1), ctypes.byref(srt), fake, 16, None) == wrs.WRS_ERR_SCRATCH
    # the refit takes the build's arguments and checks them the same way
    assert lib.wrs_refit_lbvh(ctypes.byref(big), None, 1.0, ctypes.byref(bv), ctypes.byref(srt), fake, 1 << 30, None) == wrs.WRS_ERR_ARG
    assert "wrs_refit_lbvh" in wrs.last_error()
    assert lib.wrs_refit_lbvh(ctypes.byref(big), None, 1.0, ctypes.byref(bv1), ctypes.byref(nosrc), fake, 1 << 30, None) == wrs.WRS_ERR_ARG
    assert lib.wrs_refit_lbvh(ctypes.byref(big), None, 1.0, ctypes.byref(small), ctypes.byref(srt), fake, 1 << 30, None) == wrs.WRS_ERR_CAPACITY
    assert lib.wrs_refit_lbvh(ctypes.byref(big), None, 1.0, ctypes.byref(bv1), ctypes.byref(srt), fake, 16, None) == wrs.WRS_ERR_SCRATCH
    assert lib.wrs_refit_lbvh(ctypes.byref(big), None, float("nan"), ctypes.byref(bv1), ctypes.byref(srt), fake, 1 << 30, None) == wrs.WRS_ERR_ARG
    # trace: bad k_chunk / block / t_stop / edge softness
    for p in (wrs._Params(0, 1e-5, 0.0, None, 3, 128), wrs._Params(0, 1e-5, 0.0, None, 8, 96),
              wrs._Params(0, 1.5, 0.0, None, 8, 128), wrs._Params(0, 1e-5, 1.0, None, 8, 128),
              wrs._Params(-1, 1e-5, 0.0, None, 8, 128)):
        assert lib.wrs_trace(ctypes.byref(bv1), ctypes.byref(srt), ctypes.byref(_cam(wrs)), ctypes.byref(p), fake, None, None) == wrs.WRS_ERR_ARG
    # misaligned output
    p = wrs._Params(0, 1e-5, 0.0, None, 8, 128)
    assert lib.wrs_trace(ctypes.byref(bv1), ctypes.byref(srt), ctypes.byref(_cam(wrs)), ctypes.byref(p), ctypes.c_void_p(0x1004), None, None) == wrs.WRS_ERR_ARG
    # several views: none, a view of another size, a bad camera, a misaligned gradient image
    cams = (wrs.Camera * 3)(_cam(wrs), _cam(wrs), _cam(wrs, w=9))
    assert lib.wrs_trace_views(ctypes.byref(bv1), ctypes.byref(srt), cams, 0, ctypes.byref(p), fake, None, None) == wrs.WRS_ERR_ARG
    assert lib.wrs_trace_views(ctypes.byref(bv1), ctypes.byref(srt), None, 2, ctypes.byref(p), fake, None, None) == wrs.WRS_ERR_ARG
    assert lib.wrs_trace_views(ctypes.byref(bv1), ctypes.byref(srt), cams, 3, ctypes.byref(p), fake, None, None) == wrs.WRS_ERR_ARG
    assert "view 2 is 9x8" in wrs.last_error()
    cams[1].tan_half_fovy = 0.0
    assert lib.wrs_trace_views(ctypes.byref(bv1), ctypes.byref(srt), cams, 2, ctypes.byref(p), fake, None, None) == wrs.WRS_ERR_ARG
    cams[1].tan_half_fovy = 0.4
    assert lib.wrs_trace_backward_views(ctypes.byref(bv1), ctypes.byref(srt), cams, 3, ctypes.byref(p), None, 1.0, fake, fake, None, None, 0, None, None) == wrs.WRS_ERR_ARG
    assert lib.wrs_trace_backward_views(ctypes.byref(bv1), ctypes.byref(srt), cams, 2, ctypes.byref(p), None, 1.0, ctypes.c_void_p(0x1004), fake, None, None, 0, None, None) == wrs.WRS_ERR_ARG
    # batched: no sessions; an unknown schedule.  The per-session schedule is batched-only.
    assert lib.wrs_trace_batched(fake, 0, 0, ctypes.byref(p), fake, None, None) == wrs.WRS_ERR_ARG
    ps = wrs._Params(0, 1e-5, 0.0, None, 1, 128, 4, 4)
    assert lib.wrs_trace_batched(fake, 1, 1, ctypes.byref(ps), fake, None, None) == wrs.WRS_ERR_ARG
    assert "unknown schedule 4" in wrs.last_error()
    ps.schedule = wrs.SCHEDULE_PER_SESSION
    assert lib.wrs_trace(ctypes.byref(bv1), ctypes.byref(srt), ctypes.byref(_cam(wrs)), ctypes.byref(ps), fake, None, None) == wrs.WRS_ERR_ARG
    # measurement helpers: no output, no blocks or repetitions, misaligned or odd-sized copies
    assert lib.wrs_fma_peak(None, 4, 10, None) == wrs.WRS_ERR_ARG
    assert lib.wrs_fma_peak(fake, 0, 10, None) == wrs.WRS_ERR_ARG
    assert lib.wrs_stream_copy(fake, fake, 24, 4, 1, None) == wrs.WRS_ERR_ARG
    assert lib.wrs_stream_copy(fake, ctypes.c_void_p(0x1008), 32, 4, 1, None) == wrs.WRS_ERR_ARG
    assert lib.wrs_stream_copy(fake, fake, 32, 4, 0, None) == wrs.WRS_ERR_ARG
    # ray caster: bad dtype, bad size
    assert lib.wrs_raycast_volume(fake, 5, 4, 4, 4, fake, ctypes.byref(_cam(wrs)), 0.5, 0.1, fake, fake, None) == wrs.WRS_ERR_ARG
    assert lib.wrs_raycast_volume(fake, 0, 0, 4, 4, fake, ctypes.byref(_cam(wrs)), 0.5, 0.1, fake, fake, None) == wrs.WRS_ERR_ARG
    assert lib.wrs_check_status(None, None) == wrs.WRS_ERR_ARG


def test_tree_layout_checks_without_device(wrs):
    """The 4-wide-only layout (WRS_LBVH_WIDE): the binding's constants are the header's; an
    unknown layout is refused by the build, the refit and the traces; the binary traversal (width
    2 or 0 under any schedule but the packet one) of such a tree is refused before any CUDA call."""
    import re
    hdr = open(os.path.join(ROOT, "include", "wrs.h")).read()
    consts = dict(re.findall(r"#define (WRS_LBVH_\w+) (\d+)", hdr))
    assert int(consts["WRS_LBVH_FULL"]) == wrs.LBVH_FULL == 0
    assert int(consts["WRS_LBVH_WIDE"]) == wrs.LBVH_WIDE
    lib = wrs.lib
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: validation fails first
    big = wrs._Splats(fake.value, fake.value, fake.value, None, fake.value, 64)
    srt = wrs._Splats(fake.value, fake.value, fake.value, fake.value, fake.value, 64)
    odd = wrs._Lbvh(fake.value, 64, 1, 2)
    for fn in (lib.wrs_build_lbvh, lib.wrs_refit_lbvh):
        assert fn(ctypes.byref(big), None, 1.0, ctypes.byref(odd), ctypes.byref(srt), fake, 1 << 30, None) == wrs.WRS_ERR_ARG
        assert "layout 2" in wrs.last_error()
    p4 = wrs._Params(0, 1e-5, 0.0, None, 8, 128, 0, 4)
    assert lib.wrs_trace(ctypes.byref(odd), ctypes.byref(srt), ctypes.byref(_cam(wrs)), ctypes.byref(p4), fake, None, None) == wrs.WRS_ERR_ARG
    wide = wrs._Lbvh(fake.value, 64, 1, wrs.LBVH_WIDE)
    cams = (wrs.Camera * 2)(_cam(wrs), _cam(wrs))
    for width in (2, 0):
        for sched in (wrs.SCHEDULE_PER_PIXEL, wrs.SCHEDULE_PERSISTENT):
            p2 = wrs._Params(0, 1e-5, 0.0, None, 8, 128, sched, width)
            assert lib.wrs_trace(ctypes.byref(wide), ctypes.byref(srt), ctypes.byref(_cam(wrs)), ctypes.byref(p2), fake, None, None) == wrs.WRS_ERR_ARG
            assert "WRS_LBVH_FULL" in wrs.last_error()
        assert lib.wrs_trace_views(ctypes.byref(wide), ctypes.byref(srt), cams, 2, ctypes.byref(p2), fake, None, None) == wrs.WRS_ERR_ARG
        assert lib.wrs_trace_count(ctypes.byref(wide), ctypes.byref(srt), ctypes.byref(_cam(wrs)), ctypes.byref(p2), fake, None, None) == wrs.WRS_ERR_ARG
        assert lib.wrs_trace_backward_views(ctypes.byref(wide), ctypes.byref(srt), cams, 2, ctypes.byref(p2), None, 1.0, fake, fake, None, None, 0, None, None) == wrs.WRS_ERR_ARG
        assert "WRS_LBVH_FULL" in wrs.last_error()


def test_tree_layout_follows_the_traversal(wrs):
    """A trace that walks the 4-wide nodes (width 4, or the packet schedule at any width) needs
    only the 4-wide-only layout; the binary traversal needs the full one."""
    P = wrs.TraceParams
    assert wrs.tree_layout(P(width=4)) == wrs.LBVH_WIDE
    assert wrs.tree_layout(P(width=4, schedule=wrs.SCHEDULE_PERSISTENT)) == wrs.LBVH_WIDE
    assert wrs.tree_layout(P(width=2, schedule=wrs.SCHEDULE_PACKET)) == wrs.LBVH_WIDE
    for sched in (wrs.SCHEDULE_PER_PIXEL, wrs.SCHEDULE_PERSISTENT):
        for width in (0, 2):
            assert wrs.tree_layout(P(width=width, schedule=sched)) == wrs.LBVH_FULL


def test_cpu_tensors_are_rejected(wrs):
    import torch
    with pytest.raises(ValueError):
        wrs._ptr(torch.zeros(4))


def test_buffer_checks(wrs):
    """Caller buffers the kernels index by the camera's size are checked before any call (the C ABI
    takes raw pointers): dtype and element count (CPU tensors are refused as before)."""
    import torch
    with pytest.raises(ValueError, match="dtype"):
        wrs._buf(torch.zeros(8, dtype=torch.float64), 8, torch.float32, "x")
    with pytest.raises(ValueError, match="at least"):
        wrs._buf(torch.zeros(7), 8, torch.float32, "x")
    with pytest.raises(ValueError, match="CUDA"):
        wrs._buf(torch.zeros(8), 8, torch.float32, "x")
    assert wrs._buf(None, 8, torch.float32, "x") is None


def test_window_weight_is_the_oracle_power(wrs):
    """wrs_window_weight (host function) against the oracle's binary32 powers of the decay."""
    import numpy as np

    import oracle
    for decay in (1.0, 0.9, 0.75, 0.5, 0.3333):
        ref = oracle.window_weights(9, decay)
        got = np.array([wrs.window_weight(decay, g) for g in range(9)], np.float32)
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), decay
    for bad in (0.0, -0.5, 1.5, float("nan")):
        with pytest.raises(ValueError):
            wrs.window_weight(bad, 2)
