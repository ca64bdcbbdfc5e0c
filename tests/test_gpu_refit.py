"""The LBVH refit (wrs_refit_lbvh) over fixed splat centres: with new radius scales it gives bitwise
the tree, header and sorted splats of a new build (wrs_build_lbvh, which the parity tests pin to the
oracle's Karras tree), and the same images; the radius fit that uses it follows an uninterrupted
fit (tests/test_gpu_fit.py)."""
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


def _splats(wrs, w=96, h=72, seed=31):
    rgba, depth = synth.synthetic_server_image(w, h, seed, hole_frac=0.1)
    srv = synth.server_camera(1.4, 30.0, w, h)
    return wrs.unproject(torch.from_numpy(rgba).cuda(), torch.from_numpy(depth).cuda(), srv), srv


def _same_tree(wrs, a, sa, b, sb):
    """Header, binary records (boxes and references), 4-wide nodes and sorted splats equal."""
    ha, hb = a.header(), b.header()
    assert ha == hb
    m = ha["m"]
    if m > 1:
        k = m - 1
        assert torch.equal(a.nodes[64:64 + 64 * k], b.nodes[64:64 + 64 * k])
        wa, ra = a.wide_table()
        wb, rb = b.wide_table()
        assert torch.equal(wa.view(torch.int32), wb.view(torch.int32)) and torch.equal(ra, rb)
    n = sa.count()
    assert n == sb.count()
    for x, y in zip(sa.view(), sb.view()):
        assert torch.equal(x.contiguous().view(torch.int32), y.contiguous().view(torch.int32))


@pytest.mark.parametrize("leaf", [1, 2, 4])
def test_refit_equals_build(wrs, leaf):
    sp, _ = _splats(wrs)
    n = sp.count()
    g = torch.Generator(device="cpu").manual_seed(leaf)
    s1 = (0.5 + torch.rand(n, generator=g)).cuda()
    s2 = (torch.rand(n, generator=g) * 2.0 - 0.3).cuda()  # some scales <= 0: radius 0
    tree = wrs.RefitTree(sp, leaf)
    tree.update(s1)                      # the build
    bvh, srt = tree.update(s2)           # the refit
    ref_bvh, ref_srt = wrs.build_lbvh(sp, leaf, radius_scale=s2)
    _same_tree(wrs, bvh, srt, ref_bvh, ref_srt)
    # and a third set of scales after the refit, then back to the global scale
    s3 = (0.2 + torch.rand(n, generator=g) * 3.0).cuda()
    bvh, srt = tree.update(s3)
    ref_bvh, ref_srt = wrs.build_lbvh(sp, leaf, radius_scale=s3)
    _same_tree(wrs, bvh, srt, ref_bvh, ref_srt)
    bvh, srt = tree.update(None, 1.7)
    ref_bvh, ref_srt = wrs.build_lbvh(sp, leaf, global_scale=1.7)
    _same_tree(wrs, bvh, srt, ref_bvh, ref_srt)


def test_refit_images_equal_build(wrs):
    sp, srv = _splats(wrs, 128, 96, 7)
    n = sp.count()
    cams = [synth.orbit(srv, (0, 1, 0), 4.0, 80, 64), synth.orbit(srv, (1, 0, 0), -6.0, 80, 64)]
    params = wrs.TraceParams(edge_softness=0.25, k_chunk=2, width=4)
    tree = wrs.RefitTree(sp, 1)
    tree.update(torch.ones(n, device="cuda"))
    sc = torch.linspace(0.5, 1.8, n, device="cuda")
    bvh, srt = tree.update(sc)
    ref_bvh, ref_srt = wrs.build_lbvh(sp, 1, radius_scale=sc)
    a = wrs.trace_views(bvh, srt, cams, params)
    b = wrs.trace_views(ref_bvh, ref_srt, cams, params)
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))


def test_refit_empty_and_single(wrs):
    cam = synth.server_camera(1.4, 30.0, 9, 9)
    rgba = np.zeros((9, 9, 4), np.float32)
    depth = np.full((9, 9), np.inf, np.float32)
    empty = wrs.unproject(torch.from_numpy(rgba).cuda(), torch.from_numpy(depth).cuda(), cam)
    tree = wrs.RefitTree(empty, 1)
    tree.update(None, 1.0)
    bvh, srt = tree.update(None, 2.0)
    assert bvh.header()["n"] == 0 and srt.count() == 0
    rgba[4, 4] = [0.3, 0.2, 0.1, 0.6]
    depth[4, 4] = 1.0
    one = wrs.unproject(torch.from_numpy(rgba).cuda(), torch.from_numpy(depth).cuda(), cam)
    tree = wrs.RefitTree(one, 1)
    tree.update(None, 1.0)
    bvh, srt = tree.update(None, 2.0)
    ref_bvh, ref_srt = wrs.build_lbvh(one, 1, global_scale=2.0)
    _same_tree(wrs, bvh, srt, ref_bvh, ref_srt)


def test_render_views_tree_checks(wrs):
    sp, srv = _splats(wrs)
    other, _ = _splats(wrs, seed=5)
    n = sp.count()
    col = sp.rgba[:n].clone()
    cams = [synth.orbit(srv, (0, 1, 0), 4.0, 32, 32)]
    with pytest.raises(ValueError):
        wrs.render_views(sp, cams, col, None, torch.ones(n, device="cuda"),
                         tree=wrs.RefitTree(other, 1))
    with pytest.raises(ValueError):
        wrs.render_views(sp, cams, col, None, torch.ones(n, device="cuda"),
                         tree=wrs.RefitTree(sp, 2))


def test_refit_equals_build_1080p(wrs):
    """The full-size case: a 1080p server image (about 2 M splats), refitted to per-splat scales
    after a build with scale 1, against a new build: every record, 4-wide node and sorted splat."""
    rgba, depth = synth.synthetic_server_image(1920, 1080, 52)
    srv = synth.LARGE.server_cam()
    sp = wrs.unproject(torch.from_numpy(rgba).cuda(), torch.from_numpy(depth).cuda(), srv)
    n = sp.count()
    assert n > 1_500_000
    tree = wrs.RefitTree(sp, 1)
    tree.update(None, 1.0)
    g = torch.Generator(device="cpu").manual_seed(9)
    sc = (0.25 + 1.5 * torch.rand(n, generator=g)).cuda()
    bvh, srt = tree.update(sc)
    ref_bvh, ref_srt = wrs.build_lbvh(sp, 1, radius_scale=sc)
    _same_tree(wrs, bvh, srt, ref_bvh, ref_srt)
