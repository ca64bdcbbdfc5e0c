"""GPU parity of the accumulation over server frames (future work, §6; reading: spec S3a) through the
C ABI: wrs_unproject_append and the window of frames against the CPU oracle.

The splat records (positions, radii, scaled colours, ids, count) must match bitwise; images of a
window within the trace tolerance (per-pixel RGBA max abs <= 2e-3, mean abs <= 1e-4).
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


def _frames(W, H, n, seed):
    base = synth.server_camera(1.4, 30.0, W, H)
    cams = [base] + synth.poses_in_cap(base, n - 1, 12.0, seed, W, H)
    out = []
    for g in range(n):
        rgba, depth = synth.synthetic_server_image(W, H, seed + 10 * g)
        out.append((rgba, depth, cams[g]))
    return out


def _records(sp):
    pos, rgba, ids = (t.cpu().numpy() for t in sp.view())
    return pos, rgba, ids.view(np.uint32)


def _assert_same(sp, ref):
    pos, rgba, ids = _records(sp)
    assert ids.shape[0] == ref.n
    assert np.array_equal(ids, ref.id)
    assert np.array_equal(pos.view(np.uint32), ref.pos_r.view(np.uint32))
    assert np.array_equal(rgba.view(np.uint32), ref.rgba.view(np.uint32))


@pytest.mark.parametrize("decay", [1.0, 0.75])
def test_window_splats_bitwise(wrs, decay):
    """Three ragged frames (61 x 47, not a multiple of the 1024-pixel compaction tile) with
    different server poses: the union equals the oracle's accumulation record for record."""
    from paper_2006_14726_b300.accumulate import FrameWindow
    fr = _frames(61, 47, 3, 300)
    win = FrameWindow(3, 61, 47, decay=decay)
    for rgba, depth, cam in reversed(fr):  # oldest first, so the window ends newest first
        win.push(_cuda(rgba), _cuda(depth), cam)
    wrs.check_status(win.status)
    _assert_same(win.splats, oracle.accumulate(fr, decay=decay))


def test_window_slides(wrs):
    """Four pushes into a window of three: the oldest frame leaves the set."""
    from paper_2006_14726_b300.accumulate import FrameWindow
    fr = _frames(40, 30, 4, 310)
    win = FrameWindow(3, 40, 30, decay=0.5)
    for rgba, depth, cam in reversed(fr):
        win.push(_cuda(rgba), _cuda(depth), cam)
    assert len(win) == 3
    _assert_same(win.splats, oracle.accumulate(fr[:3], decay=0.5))


def test_append_capacity_overflow_sets_status(wrs):
    fr = _frames(64, 48, 2, 320)
    (ra, da, ca), (rb, db, cb) = fr
    full, _ = oracle.append_frame(None, ra, da, ca)
    full, _ = oracle.append_frame(full, rb, db, cb, weight=0.5, id_base=64 * 48)
    cap = full.n - 100
    assert cap >= 64 * 48
    sp = wrs.SplatBuffers(cap)
    st = wrs.new_status()
    wrs.unproject(_cuda(ra), _cuda(da), ca, out=sp)
    wrs.unproject_append(_cuda(rb), _cuda(db), cb, sp, weight=0.5, id_base=64 * 48, status=st)
    assert sp.count() == cap
    assert int(st.item()) == wrs.STATUS_SPLAT_OVERFLOW
    with pytest.raises(wrs.WrsError, match="splat capacity overflow"):
        wrs.check_status(st)
    ref, ovf = oracle.append_frame(oracle.append_frame(None, ra, da, ca, capacity=cap)[0], rb, db, cb,
                                   weight=0.5, id_base=64 * 48, capacity=cap)
    assert ovf
    _assert_same(sp, ref)
    # a count already above the capacity is clamped and flagged; nothing is written
    sp.n.fill_(cap + 5)
    before = sp.pos_r.clone()
    wrs.unproject_append(_cuda(rb), _cuda(db), cb, sp, id_base=64 * 48, status=st)
    assert sp.count() == cap and int(st.item()) == wrs.STATUS_SPLAT_OVERFLOW
    assert torch.equal(before, sp.pos_r)
    st.zero_()


def test_append_to_empty_equals_unproject(wrs):
    """weight 1, id_base 0 on an empty set is the plain unprojection, bit for bit; an all-hole
    frame appends nothing."""
    (rgba, depth, cam), = _frames(33, 17, 1, 330)
    a = wrs.unproject(_cuda(rgba), _cuda(depth), cam)
    b = wrs.SplatBuffers(33 * 17)
    wrs.unproject_append(_cuda(rgba), _cuda(depth), cam, b)
    for x, y in zip(a.view(), b.view()):
        assert torch.equal(x, y)
    n = b.count()
    holes = np.full((17, 33), np.inf, np.float32)
    wrs.unproject_append(_cuda(np.zeros_like(rgba)), _cuda(holes), cam, b, id_base=33 * 17)
    assert b.count() == n


def test_append_rejects_bad_arguments(wrs):
    (rgba, depth, cam), = _frames(16, 8, 1, 340)
    sp = wrs.SplatBuffers(128)
    for kw in ({"weight": 0.0}, {"weight": 1.5}, {"weight": float("nan")}):
        with pytest.raises(wrs.WrsError):
            wrs.unproject_append(_cuda(rgba), _cuda(depth), cam, sp, **kw)
    with pytest.raises(ValueError):
        wrs.unproject_append(_cuda(rgba), _cuda(depth), cam, sp, id_base=2**31 - 10)


@pytest.mark.parametrize("H", [0, 1])
def test_window_trace_full_image(wrs, H):
    """Trace of a three-frame window (128 x 96 server frames, 160 x 120 client) against the
    oracle's trace of its accumulated set, every pixel."""
    from paper_2006_14726_b300.accumulate import FrameWindow
    fr = _frames(128, 96, 3, 350)
    win = FrameWindow(3, 128, 96, decay=0.8)
    for rgba, depth, cam in reversed(fr):
        win.push(_cuda(rgba), _cuda(depth), cam)
    cli = synth.orbit(fr[0][2], (0, 1, 0), 6.0, 160, 120)
    img = win.trace(cli, wrs.TraceParams(max_hits=H, width=4))
    wrs.check_status(win.status)
    ref = oracle.trace(oracle.Scene(oracle.accumulate(fr, decay=0.8), max_hits=H), cli)
    err = np.abs(img.cpu().numpy().reshape(-1, 4).astype(np.float64) - ref["rgba"])
    assert err.max() <= 1e-5 and err.mean() <= MEAN_ABS


def test_window_1080p_sampled(wrs):
    """Full-size window: four 1920 x 1080 server frames (about 8 M splats) from poses within 12
    degrees, a 1920 x 1080 client view; the spliced set bitwise against the oracle's record count
    and ids, and 4096 sampled pixels against the oracle's trace."""
    from paper_2006_14726_b300.accumulate import FrameWindow
    fr = _frames(1920, 1080, 4, 360)
    win = FrameWindow(4, 1920, 1080, decay=0.9)
    for rgba, depth, cam in reversed(fr):
        win.push(_cuda(rgba), _cuda(depth), cam)
    ref_sp = oracle.accumulate(fr, decay=0.9)
    _assert_same(win.splats, ref_sp)
    cli = synth.orbit(fr[0][2], (0.6, 0.8, 0.0), 15.0)
    pix = np.random.default_rng(11).choice(1920 * 1080, 4096, replace=False)
    ref = oracle.trace(oracle.Scene(ref_sp), cli, pixels=pix)
    for sched, width in ((0, 4), (1, 2)):
        img = win.trace(cli, wrs.TraceParams(schedule=sched, width=width, k_chunk=1))
        wrs.check_status(win.status)
        err = np.abs(img.cpu().numpy().reshape(-1, 4)[pix].astype(np.float64) - ref["rgba"])
        assert err.max() <= MAX_ABS and err.mean() <= MEAN_ABS, (sched, width, err.max())


def test_two_slot_window_overlapped_streams(wrs):
    """A window with two copies of its set, pushed on one stream and traced on another while the
    previous frame's views still trace: each step's views equal a one-copy window's bitwise, and
    the current set equals the oracle's accumulation record for record."""
    from paper_2006_14726_b300.accumulate import FrameWindow
    fr = _frames(64, 48, 6, 330)
    one = FrameWindow(3, 64, 48, decay=0.5)
    two = FrameWindow(3, 64, 48, decay=0.5, slots=2, layout=wrs.LBVH_WIDE)
    build, draw = torch.cuda.Stream(priority=-1), torch.cuda.Stream()
    cams = [synth.orbit(fr[0][2], (0, 1, 0), a, 56, 40) for a in (2.0, -3.0, 5.0)]
    p = wrs.TraceParams(k_chunk=2, width=4)
    frames_in = [(_cuda(r), _cuda(d), c) for r, d, c in reversed(fr)]
    # every output allocated up front: a buffer the allocator hands out again on the default
    # stream could still be in use there when the draw stream writes it
    ref_imgs = [[torch.empty(40, 56, 4, device="cuda") for _ in cams] for _ in frames_in]
    imgs = [[torch.empty(40, 56, 4, device="cuda") for _ in cams] for _ in frames_in]
    torch.cuda.synchronize()
    for (rgba, depth, cam), ref_o, outs in zip(frames_in, ref_imgs, imgs):
        one.push(rgba, depth, cam)
        for c, o in zip(cams, ref_o):
            one.trace(c, p, out=o)
        two.push(rgba, depth, cam, stream=build)  # overlaps the previous frame's views
        for c, o in zip(cams, outs):
            two.trace(c, p, out=o, stream=draw)
    torch.cuda.synchronize()
    wrs.check_status(two.status)
    for a, b in zip(ref_imgs, imgs):
        for x, y in zip(a, b):
            assert torch.equal(x.view(torch.int32), y.view(torch.int32))
    _assert_same(two.splats, oracle.accumulate(fr[:3], decay=0.5))
    # pushes with no trace between them, alternating streams: each rebuild also waits for the
    # last build of the copy it overwrites
    for i, (rgba, depth, cam) in enumerate(frames_in):
        two.push(rgba, depth, cam, stream=build if i % 2 else None)
    torch.cuda.synchronize()
    wrs.check_status(two.status)
    _assert_same(two.splats, oracle.accumulate(fr[:3], decay=0.5))
