"""The 4-wide-only tree layout (WRS_LBVH_WIDE): a build or refit that skips the binary records of
the nodes inside one refit block gives bitwise the 4-wide nodes, header and sorted splats of the
full layout (whose every record and 4-wide node the parity tests pin to the oracle's tree), and
the same images; the binary traversal of such a tree is refused (single trees on the host,
batched sessions through the status word)."""
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


def _splats(wrs, w=133, h=97, seed=31):
    rgba, depth = synth.synthetic_server_image(w, h, seed, hole_frac=0.1)
    srv = synth.server_camera(1.4, 30.0, w, h)
    return wrs.unproject(torch.from_numpy(rgba).cuda(), torch.from_numpy(depth).cuda(), srv), srv


def _same_wide(wrs, full, sf, wide, sw):
    """Header (but the layout word), 4-wide nodes and sorted splats bitwise equal."""
    hf, hw = full.header(), wide.header()
    assert hf.pop("layout") == wrs.LBVH_FULL and hw.pop("layout") == wrs.LBVH_WIDE
    assert hf == hw
    if hf["m"] > 1:
        bf, rf = full.wide_table()
        bw, rw = wide.wide_table()
        assert torch.equal(bf.view(torch.int32), bw.view(torch.int32)) and torch.equal(rf, rw)
    assert sf.count() == sw.count()
    for x, y in zip(sf.view(), sw.view()):
        assert torch.equal(x.contiguous().view(torch.int32), y.contiguous().view(torch.int32))


@pytest.mark.parametrize("leaf", [1, 2, 4])
def test_wide_layout_equals_full(wrs, leaf):
    sp, srv = _splats(wrs)
    n = sp.count()
    sc = (0.3 + torch.rand(n, generator=torch.Generator().manual_seed(leaf))).cuda()
    full, sf = wrs.build_lbvh(sp, leaf, radius_scale=sc)
    wide, sw = wrs.build_lbvh(sp, leaf, radius_scale=sc, layout=wrs.LBVH_WIDE)
    _same_wide(wrs, full, sf, wide, sw)
    cams = [synth.orbit(srv, (0, 1, 0), 5.0, 72, 55), synth.orbit(srv, (1, 0, 0), -7.0, 64, 48)]
    for sched in (wrs.SCHEDULE_PER_PIXEL, wrs.SCHEDULE_PERSISTENT, wrs.SCHEDULE_PACKET):
        p = wrs.TraceParams(k_chunk=4, schedule=sched, width=4)
        for c in cams:
            a = wrs.trace(full, sf, c, p)
            b = wrs.trace(wide, sw, c, p)
            assert torch.equal(a.view(torch.int32), b.view(torch.int32))
    # the packet schedule walks the 4-wide nodes whatever the width says
    p = wrs.TraceParams(k_chunk=4, schedule=wrs.SCHEDULE_PACKET, width=2)
    assert torch.equal(wrs.trace(wide, sw, cams[0], p).view(torch.int32),
                       wrs.trace(full, sf, cams[0], p).view(torch.int32))
    # the binary traversal needs the full layout
    for sched in (wrs.SCHEDULE_PER_PIXEL, wrs.SCHEDULE_PERSISTENT):
        with pytest.raises(wrs.WrsError, match="WRS_LBVH_FULL"):
            wrs.trace(wide, sw, cams[0], wrs.TraceParams(schedule=sched, width=2))


def test_wide_layout_over_stale_buffers(wrs):
    """A 4-wide-only build into buffers that held another tree: the 4-wide nodes and images are
    those of a build into fresh buffers (the records it skips are never read)."""
    sp, srv = _splats(wrs, 96, 72, 3)
    other, _ = _splats(wrs, 96, 72, 11)
    bvh = wrs.LBVH(sp.capacity, 1, layout=wrs.LBVH_WIDE)
    srt = wrs.SplatBuffers(sp.capacity, sorted=True)
    wrs.build_lbvh(other, 1, bvh=bvh, sorted=srt)
    wrs.build_lbvh(sp, 1, bvh=bvh, sorted=srt)
    full, sf = wrs.build_lbvh(sp, 1)
    _same_wide(wrs, full, sf, bvh, srt)


def test_wide_layout_refit(wrs):
    sp, _ = _splats(wrs, 96, 72, 5)
    n = sp.count()
    g = torch.Generator().manual_seed(4)
    s1 = (0.5 + torch.rand(n, generator=g)).cuda()
    s2 = (torch.rand(n, generator=g) * 2.0 - 0.3).cuda()
    tree = wrs.RefitTree(sp, 1, layout=wrs.LBVH_WIDE)
    tree.update(s1)
    bvh, srt = tree.update(s2)
    full, sf = wrs.build_lbvh(sp, 1, radius_scale=s2)
    _same_wide(wrs, full, sf, bvh, srt)


def test_wide_layout_empty_and_single(wrs):
    cam = synth.server_camera(1.4, 30.0, 9, 9)
    rgba = np.zeros((9, 9, 4), np.float32)
    depth = np.full((9, 9), np.inf, np.float32)
    for hits in (0, 1, 2):
        if hits:
            rgba[4, 3 + hits] = [0.3, 0.2, 0.1, 0.6]
            depth[4, 3 + hits] = 1.0
        sp = wrs.unproject(torch.from_numpy(rgba).cuda(), torch.from_numpy(depth).cuda(), cam)
        full, sf = wrs.build_lbvh(sp, 1)
        wide, sw = wrs.build_lbvh(sp, 1, layout=wrs.LBVH_WIDE)
        _same_wide(wrs, full, sf, wide, sw)
        p = wrs.TraceParams(width=4)
        assert torch.equal(wrs.trace(full, sf, cam, p), wrs.trace(wide, sw, cam, p))


def test_wide_layout_1080p(wrs):
    """The full-size case: a 1080p server image (about 2 M splats), both layouts, every 4-wide
    node and sorted splat; one client view's image."""
    rgba, depth = synth.synthetic_server_image(1920, 1080, 52)
    srv = synth.LARGE.server_cam()
    sp = wrs.unproject(torch.from_numpy(rgba).cuda(), torch.from_numpy(depth).cuda(), srv)
    assert sp.count() > 1_500_000
    full, sf = wrs.build_lbvh(sp, 1)
    wide, sw = wrs.build_lbvh(sp, 1, layout=wrs.LBVH_WIDE)
    _same_wide(wrs, full, sf, wide, sw)
    cam = synth.LARGE.client_poses()[1]
    p = wrs.TraceParams(k_chunk=1, width=4)
    assert torch.equal(wrs.trace(full, sf, cam, p).view(torch.int32),
                       wrs.trace(wide, sw, cam, p).view(torch.int32))


def test_batched_wide_sessions(wrs):
    """Sessions over 4-wide-only trees: traced 4-wide, their images equal the full trees'; traced
    over binary nodes, the status word reports a malformed tree (the images are undefined)."""
    sess_w, sess_f = [], []
    for s in range(3):
        sp, srv = _splats(wrs, 64 + 16 * s, 48 + 8 * s, 40 + s)
        cam = synth.orbit(srv, (0, 1, 0), 3.0 + s, 40 + 8 * s, 32)
        b, so = wrs.build_lbvh(sp, 1, layout=wrs.LBVH_WIDE)
        sess_w.append((b, so, cam))
        sess_f.append(wrs.build_lbvh(sp, 1) + (cam,))
    bw, bf = wrs.Batch(sess_w), wrs.Batch(sess_f)
    for sched in (wrs.SCHEDULE_PER_PIXEL, wrs.SCHEDULE_PACKET, wrs.SCHEDULE_PER_SESSION,
                  wrs.SCHEDULE_PERSISTENT):
        p = wrs.TraceParams(k_chunk=2, schedule=sched, width=4)
        st = wrs.new_status()
        ow = [o.clone() for o in wrs.trace_batched(bw, p, status=st)]
        of = wrs.trace_batched(bf, p)
        wrs.check_status(st)
        for a, b in zip(ow, of):
            assert torch.equal(a.view(torch.int32), b.view(torch.int32))
    for sched in (wrs.SCHEDULE_PER_PIXEL, wrs.SCHEDULE_PERSISTENT):
        st = wrs.new_status()
        wrs.trace_batched(bw, wrs.TraceParams(k_chunk=2, schedule=sched, width=2), status=st)
        torch.cuda.synchronize()
        assert int(st.item()) & wrs.STATUS_MALFORMED_TREE
    # sessions traced by their own (packet) schedule walk the 4-wide nodes: no error
    bp = wrs.Batch(sess_w, schedules=[wrs.SCHEDULE_PACKET] * 3)
    st = wrs.new_status()
    wrs.trace_batched(bp, wrs.TraceParams(k_chunk=2, schedule=wrs.SCHEDULE_PER_SESSION, width=2),
                      status=st)
    wrs.check_status(st)
