"""Recorded hit lists (wrs_trace_views_record) and the adjoint from them without traversal
(wrs_trace_backward_views_recorded), through the C ABI.

The forward images equal the plain multi-view trace bitwise; every complete list holds exactly
the oracle's composited hits in order (the oracle's FNV-1a hash of their ids per pixel); lists
over capacity are marked and their rays re-traversed; the gradients equal the re-traversing
adjoint's up to the order of the float atomics, and the oracle adjoint element by element at the
differentiation workload's size (tests/test_gpu_backward.py's tolerance)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FNV_OFFSET = 1469598103934665603
FNV_PRIME = 1099511628211


@pytest.fixture(scope="module")
def wrs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_14726_b300 as w
    oracle.build()
    return w


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _instance(wrs, seed=44):
    rgba, depth = synth.synthetic_server_image(96, 72, seed, hole_frac=0.1)
    srv = synth.server_camera(1.4, 30.0, 96, 72)
    ref_sp = oracle.unproject(rgba, depth, srv)
    sp = wrs.unproject(_cuda(rgba), _cuda(depth), srv)
    cams = [synth.orbit(srv, (0, 1, 0), 2.0 + 3 * v, 80, 64) for v in range(4)]
    rng = np.random.default_rng(seed)
    sc = rng.uniform(1.0, 2.5, ref_sp.n).astype(np.float32)
    op = rng.uniform(0.3, 1.0, ref_sp.n).astype(np.float32)
    return sp, ref_sp, cams, sc, op


def _fnv(ids):
    h = FNV_OFFSET
    for i in ids:
        h = ((h ^ int(i)) * FNV_PRIME) & 0xFFFFFFFFFFFFFFFF
    return h


@pytest.mark.parametrize("sched,k,cap", [(0, 2, 16), (2, 4, 16), (0, 4, 16), (0, 1, 3), (2, 4, 2)])
def test_record_images_and_lists(wrs, sched, k, cap):
    sp, ref_sp, cams, sc, op = _instance(wrs)
    bvh, srt = wrs.build_lbvh(sp, 1, radius_scale=_cuda(sc))
    params = wrs.TraceParams(edge_softness=0.25, k_chunk=k, schedule=sched, width=4)
    st = wrs.new_status()
    plain = wrs.trace_views(bvh, srt, cams, params, opacity=_cuda(op))
    imgs, lists = wrs.trace_views_record(bvh, srt, cams, params, cap, opacity=_cuda(op), status=st)
    wrs.check_status(st)
    assert torch.equal(imgs.view(torch.int32), plain.view(torch.int32))
    hits = lists.hits.cpu().numpy().view(np.uint32)
    count = lists.count.cpu().numpy().view(np.uint32)
    sid = srt.id.cpu().numpy().view(np.uint32)
    npix = cams[0].width * cams[0].height
    scene = oracle.Scene(ref_sp, scale=sc, opacity=op, beta=0.25)
    over = 0
    for v, cam in enumerate(cams):
        ref = oracle.trace(scene, cam)
        for p in range(npix):
            r = v * npix + p
            if count[r] > cap:
                assert count[r] == cap + 1 and ref["nused"][p] > cap
                over += 1
                continue
            assert count[r] == ref["nused"][p]
            assert _fnv(sid[hits[r, :count[r]]]) == int(ref["hash"][p]), (v, p)
    if cap <= 3:
        assert over > 0  # the capacity is exceeded and marked
    else:
        assert over < 0.01 * len(cams) * npix  # a few deep pixels only


@pytest.mark.parametrize("sched,k,cap", [(0, 2, 16), (2, 4, 16), (0, 4, 16), (2, 4, 2), (0, 1, 1)])
def test_recorded_adjoint_equals_retraversal(wrs, sched, k, cap):
    sp, ref_sp, cams, sc, op = _instance(wrs, 45)
    n = ref_sp.n
    bvh, srt = wrs.build_lbvh(sp, 1, radius_scale=_cuda(sc))
    params = wrs.TraceParams(edge_softness=0.25, k_chunk=k, schedule=sched, width=4)
    _, lists = wrs.trace_views_record(bvh, srt, cams, params, cap, opacity=_cuda(op))
    g = torch.randn(len(cams), cams[0].height, cams[0].width, 4, device="cuda")
    st = wrs.new_status()
    a = wrs.trace_backward_views_recorded(bvh, srt, cams, lists, g, params, opacity=_cuda(op),
                                          radius_scale=_cuda(sc), status=st)
    wrs.check_status(st)
    b = wrs.trace_backward_views(bvh, srt, cams, g, params, opacity=_cuda(op), radius_scale=_cuda(sc))
    for x, y in zip(a, b):
        assert torch.allclose(x[:n], y[:n], rtol=1e-4, atol=1e-5)
    # accumulate: a second view set added on top
    acc = tuple(t.clone() for t in a)
    wrs.trace_backward_views_recorded(bvh, srt, cams, lists, g, params, opacity=_cuda(op),
                                      radius_scale=_cuda(sc), accumulate_into=acc)
    for x, y in zip(acc, a):
        assert torch.allclose(x[:n], 2 * y[:n], rtol=1e-4, atol=1e-5)


def test_render_views_records_by_default(wrs):
    sp, ref_sp, cams, sc, op = _instance(wrs, 46)
    n = ref_sp.n
    params = wrs.TraceParams(edge_softness=0.25, k_chunk=2, width=4)
    grads = []
    for rec in (None, 0):
        col = sp.rgba[:n].clone().requires_grad_(True)
        opa = _cuda(op).requires_grad_(True)
        scl = _cuda(sc).requires_grad_(True)
        imgs = wrs.render_views(sp, cams, col, opa, scl, params, 1, record_hits=rec)
        g = torch.Generator(device="cuda").manual_seed(5)
        (imgs * torch.randn(imgs.shape, device="cuda", generator=g)).sum().backward()
        grads.append((imgs.detach(), col.grad, opa.grad, scl.grad))
    assert torch.equal(grads[0][0], grads[1][0])
    for x, y in zip(grads[0][1:], grads[1][1:]):
        assert torch.allclose(x, y, rtol=1e-4, atol=1e-5)


def test_recording_argument_checks(wrs):
    sp, ref_sp, cams, sc, op = _instance(wrs)
    bvh, srt = wrs.build_lbvh(sp, 1)
    with pytest.raises(ValueError):
        wrs.HitLists(10, 0)
    with pytest.raises(ValueError):
        wrs.HitLists(10, 33)
    lists = wrs.HitLists(7, 4)
    with pytest.raises(ValueError):
        wrs.trace_views_record(bvh, srt, cams, wrs.TraceParams(), lists=lists)
