"""Several client views of one scene in one launch (wrs_trace_views, wrs_trace_backward_views)
against the single-view calls, which the parity tests pin to the oracle, and directly against the
oracle on a small case.

Forward: each view is bitwise the image of its own wrs_trace call, for every schedule, width and
K, also when the views are split over several launches (more than 32 views).  Backward (one thread
per pixel, and the packet backward with a warp-shared traversal): the sum of the single-view
gradients, up to the summation order of float atomics.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_ABS = 2e-3
MEAN_ABS = 1e-4


def _same_sum(a, b):
    """a and b hold the same float32 sums accumulated by atomics in different orders.  An element
    sums the contributions of every hit of every view, of both signs (random upstream gradients),
    so its rounding error is a few ulp of its largest contributions, not of the (often much
    smaller) sum: the absolute tolerance is relative to the largest element of the buffer."""
    scale = float(b.abs().max()) if b.numel() else 0.0
    return torch.allclose(a, b, rtol=1e-4, atol=max(1e-5 * scale, 1e-7))


@pytest.fixture(scope="module")
def wrs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_14726_b300 as w
    oracle.build()
    return w


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _scene(wrs, w=96, h=72, seed=44, radius_scale=None):
    rgba, depth = synth.synthetic_server_image(w, h, seed, hole_frac=0.1)
    srv = synth.server_camera(1.4, 30.0, w, h)
    sp = wrs.unproject(_cuda(rgba), _cuda(depth), srv)
    return rgba, depth, srv, sp


def _views(srv, n, w=80, h=64):
    # orbits about two axes, 0.5 to ~12 degrees: rays that hit, graze and miss
    return [synth.orbit(srv, (0, 1, 0) if v % 2 == 0 else (1, 0, 0), 0.5 + 0.35 * v, w, h)
            for v in range(n)]


@pytest.mark.parametrize("sched,width,k", [(0, 4, 1), (0, 2, 4), (1, 4, 2), (2, 4, 1), (2, 4, 4),
                                           (0, 4, 16)])
def test_views_equal_single_view_traces_bitwise(wrs, sched, width, k):
    _, _, srv, sp = _scene(wrs)
    bvh, srt = wrs.build_lbvh(sp, 2)
    cams = _views(srv, 5)
    params = wrs.TraceParams(max_hits=0, k_chunk=k, schedule=sched, width=width,
                             edge_softness=0.25 if k > 1 else 0.0)
    st = wrs.new_status()
    imgs = wrs.trace_views(bvh, srt, cams, params, status=st)
    wrs.check_status(st)
    assert imgs.shape == (5, 64, 80, 4)
    for v, c in enumerate(cams):
        one = wrs.trace(bvh, srt, c, params)
        assert torch.equal(imgs[v], one), v


def test_more_views_than_one_launch_holds(wrs):
    """35 views: two launches (32 + 3); ragged image size (not a multiple of the 16-pixel block
    width or the block height)."""
    _, _, srv, sp = _scene(wrs, 64, 48, 7)
    bvh, srt = wrs.build_lbvh(sp, 1)
    cams = _views(srv, 35, 37, 29)
    params = wrs.TraceParams(k_chunk=1, width=4)
    imgs = wrs.trace_views(bvh, srt, cams, params)
    for v in (0, 31, 32, 34):
        assert torch.equal(imgs[v], wrs.trace(bvh, srt, cams[v], params)), v


def test_views_against_the_oracle(wrs):
    rgba, depth, srv, sp = _scene(wrs, 48, 36, 12)
    ref_sp = oracle.unproject(rgba, depth, srv)
    bvh, srt = wrs.build_lbvh(sp, 1)
    cams = _views(srv, 3, 40, 30)
    imgs = wrs.trace_views(bvh, srt, cams, wrs.TraceParams(k_chunk=2, width=4)).cpu().numpy()
    for v, c in enumerate(cams):
        want = oracle.trace(oracle.Scene(ref_sp), c)["rgba"]
        err = np.abs(imgs[v].reshape(-1, 4).astype(np.float64) - want)
        assert err.max() <= MAX_ABS and err.mean() <= MEAN_ABS, (v, err.max())


@pytest.mark.parametrize("k,width,sched", [(1, 4, 0), (4, 2, 0), (2, 4, 0), (4, 4, 2), (1, 4, 2)])
def test_backward_views_sum_the_single_view_gradients(wrs, k, width, sched):
    _, _, srv, sp = _scene(wrs)
    n = sp.count()
    scale = torch.full((n,), 1.3, device="cuda")
    opac = torch.full((n,), 0.8, device="cuda")
    bvh, srt = wrs.build_lbvh(sp, 1, radius_scale=scale)
    cams = _views(srv, 4)
    params = wrs.TraceParams(edge_softness=0.25, k_chunk=k, width=width, schedule=sched)
    g = torch.randn(len(cams), 64, 80, 4, device="cuda")
    st = wrs.new_status()
    gr, go, gs = wrs.trace_backward_views(bvh, srt, cams, g, params, opacity=opac,
                                          radius_scale=scale, status=st)
    wrs.check_status(st)
    acc = tuple(torch.zeros_like(t) for t in (gr, go, gs))
    for v, c in enumerate(cams):
        wrs.trace_backward(bvh, srt, c, g[v], params, opacity=opac, radius_scale=scale,
                           accumulate_into=acc)
    for a, b in zip((gr, go, gs), acc):
        assert _same_sum(a[:n], b[:n])
    assert float(gs[:n].abs().sum()) > 0  # the soft edges give the radius a gradient
    # accumulate = 1 adds to the buffers: twice the gradient
    wrs.trace_backward_views(bvh, srt, cams, g, params, opacity=opac, radius_scale=scale,
                             accumulate_into=(gr, go, gs))
    for a, b in zip((gr, go, gs), acc):
        assert _same_sum(a[:n], 2 * b[:n])


@pytest.mark.parametrize("sched", [0, 2])
def test_backward_over_more_views_than_one_launch_holds(wrs, sched):
    """35 ragged views (two launches of 32 + 3): the sum of the 35 single-view gradients."""
    _, _, srv, sp = _scene(wrs, 64, 48, 9)
    n = sp.count()
    bvh, srt = wrs.build_lbvh(sp, 1)
    cams = _views(srv, 35, 37, 29)
    params = wrs.TraceParams(edge_softness=0.25, k_chunk=2, width=4, schedule=sched)
    g = torch.randn(len(cams), 29, 37, 4, device="cuda")
    gr, go, _ = wrs.trace_backward_views(bvh, srt, cams, g, params, want_scale=False)
    acc = (torch.zeros_like(gr), torch.zeros_like(go), None)
    for v, c in enumerate(cams):
        wrs.trace_backward(bvh, srt, c, g[v], params, accumulate_into=acc)
    assert _same_sum(gr[:n], acc[0][:n])
    assert _same_sum(go[:n], acc[1][:n])


@pytest.mark.parametrize("k", [1, 4, 16])
def test_packet_backward_equals_per_pixel_backward(wrs, k):
    """The warp-shared traversal of the packet backward rebuilds each ray's own hit lists: its
    gradients equal the per-pixel backward's up to the order of the float atomics."""
    _, _, srv, sp = _scene(wrs, 96, 72, 21)
    n = sp.count()
    scale = torch.full((n,), 1.4, device="cuda")
    bvh, srt = wrs.build_lbvh(sp, 1, radius_scale=scale)
    cam = _views(srv, 2)[1]
    g = torch.randn(64, 80, 4, device="cuda")
    res = []
    for sched in (0, 2):
        st = wrs.new_status()
        res.append(wrs.trace_backward(bvh, srt, cam, g, wrs.TraceParams(edge_softness=0.25,
                                      k_chunk=k, width=4, schedule=sched), radius_scale=scale,
                                      status=st))
        wrs.check_status(st)
    for a, b in zip(*res):
        assert float(b[:n].abs().sum()) > 0
        assert _same_sum(a[:n], b[:n])


def test_views_of_different_sizes_are_rejected(wrs):
    _, _, srv, sp = _scene(wrs, 32, 24, 3)
    bvh, srt = wrs.build_lbvh(sp, 1)
    cams = [synth.orbit(srv, (0, 1, 0), 2.0, 40, 30), synth.orbit(srv, (0, 1, 0), 3.0, 41, 30)]
    with pytest.raises(wrs.WrsError):
        wrs.trace_views(bvh, srt, cams)
