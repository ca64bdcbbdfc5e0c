"""GPU adjoint of the ordered compositing (spec S7; not in the paper, motivated by fitting the
radius to data, §6) against the binary64 oracle adjoint and against central finite differences,
element by element, through the C ABI.

Tolerance, per gradient element g (each parameter group: RGBA, opacity, radius scale):

    |g_gpu - g_ref| <= RTOL * |g_ref| + ATOL * max|g_ref|

with RTOL = 1e-3 and ATOL = 1e-4.  Each element is a sum over the hits that reach the splat of
terms evaluated in binary32 (a chain of some tens of roundings: relative error below 3e-6 each)
and accumulated by float atomics in any order (at most one rounding per term of the running
sum), so the error is below about 1e-5 of the sum of the terms' magnitudes; terms of opposite
sign make that sum larger than |g| itself, which the ATOL part covers up to a sum of ten times
the largest gradient.  With a soft edge the distance of the ray from a centre is binary32
(relative error near 1e-5 at the rim) and enters the weight's derivative, whose slope is at
most 6 / beta^2 = 96 at beta = 0.25: about 1e-3 relative on rim terms of the scale gradient,
hence RTOL.  The radius-scale group has a larger absolute part, ATOL_SCALE = 2e-3: the binary32
ratio rho = |f| / r is off by up to about 5 ulp of the eye-to-centre distance over r (|f| is
the small residual of two binary32 vectors of length |oc|), 4e-4 at the differentiation
workload (eye 1.4 away, r near 1e-3), so the weight's derivative (slope at most 96) is off by up
to 0.04 against its largest value 1.5 / beta = 6: 0.6 % of the largest scale term in the worst
case, a few tenths of that typically (as in the images).

Cases: the 64x64 instance (every schedule, K and node width), the autograd Function, the
differentiation workload's size (512^2 server image of the 256^3 volume, 262,144 splats, one
512^2 view and all 8 views in one launch, beta = 0.25) and the GPU gradient against central
finite differences (h = 1e-3) of the GPU forward on the 64x64 / 4,096-splat instance.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-3
ATOL = 1e-4
ATOL_SCALE = 2e-3


@pytest.fixture(scope="module")
def wrs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_14726_b300 as w
    oracle.build()
    return w


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def assert_elementwise(got, ref, what, rtol=RTOL, atol=ATOL):
    got = np.asarray(got, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    scale = max(float(np.abs(ref).max()), 1e-30)
    err = np.abs(got - ref)
    bound = rtol * np.abs(ref) + atol * scale
    ratio = err / bound
    worst = int(np.argmax(ratio))
    print(f"{what}: {ref.size} elements, worst err/bound {ratio[worst]:.3f} "
          f"(element {worst}: gpu {got[worst]:.6g} ref {ref[worst]:.6g}), max |ref| {scale:.3g}")
    bad = np.flatnonzero(err > bound)
    assert bad.size == 0, f"{what}: {bad.size} elements out of tolerance, first {bad[:8].tolist()}"


def _bwd_instance(W=64, H=64, seed=0, hole_frac=0.1):
    rgba, depth = synth.synthetic_server_image(W, H, seed, hole_frac=hole_frac)
    srv = synth.server_camera(1.4, 30.0, W, H)
    ref_sp = oracle.unproject(rgba, depth, srv)
    n = ref_sp.n
    rng = np.random.default_rng(seed)
    op = rng.uniform(0.3, 1.0, n).astype(np.float32)
    sc = rng.uniform(1.0, 2.5, n).astype(np.float32)
    cli = synth.orbit(srv, (0.3, 1.0, 0.0), 10.0)
    g = rng.normal(size=(cli.width * cli.height, 4)).astype(np.float32)
    return rgba, depth, srv, cli, ref_sp, op, sc, g


@pytest.mark.parametrize("beta,k,sched,width", [(0.25, 8, 0, 2), (0.25, 1, 0, 4), (0.0, 4, 0, 2),
                                                (0.25, 1, 1, 2), (0.25, 4, 1, 4), (0.0, 2, 1, 4),
                                                (0.25, 4, 2, 4), (0.0, 1, 2, 4), (0.25, 16, 2, 4)])
def test_backward_matches_oracle_adjoint(wrs, beta, k, sched, width):
    rgba, depth, srv, cli, ref_sp, op, sc, g = _bwd_instance()
    n = ref_sp.n
    sp = wrs.unproject(_cuda(rgba), _cuda(depth), srv)
    bvh, srt = wrs.build_lbvh(sp, 1, radius_scale=_cuda(sc))
    params = wrs.TraceParams(edge_softness=beta, k_chunk=k, schedule=sched, width=width)
    st = wrs.new_status()
    gr, go, gs = wrs.trace_backward(bvh, srt, cli, _cuda(g.reshape(cli.height, cli.width, 4)),
                                    params, opacity=_cuda(op), radius_scale=_cuda(sc), status=st)
    wrs.check_status(st)
    scene = oracle.Scene(ref_sp, scale=sc, opacity=op, beta=beta)
    rr, ro, rs = oracle.trace_backward(scene, cli, g.astype(np.float64))
    what = f"beta={beta} K={k} schedule={sched} width={width}"
    assert_elementwise(gr.cpu().numpy()[:n], rr, f"{what} rgba")
    assert_elementwise(go.cpu().numpy()[:n], ro, f"{what} opacity")
    if beta > 0:
        assert np.abs(rs).max() > 0
        assert_elementwise(gs.cpu().numpy()[:n], rs, f"{what} scale", atol=ATOL_SCALE)
    else:
        assert np.all(gs.cpu().numpy()[:n] == 0)


def test_autograd_function_matches_oracle(wrs):
    rgba, depth, srv, cli, ref_sp, op, sc, g = _bwd_instance(48, 40, 3)
    sp = wrs.unproject(_cuda(rgba), _cuda(depth), srv)
    col = torch.tensor(ref_sp.rgba, device="cuda", requires_grad=True)
    opt = torch.tensor(op, device="cuda", requires_grad=True)
    sct = torch.tensor(sc, device="cuda", requires_grad=True)
    params = wrs.TraceParams(edge_softness=0.25)
    img = wrs.render(sp, cli, col, opt, sct, params)
    gt = _cuda(g.reshape(cli.height, cli.width, 4))
    (img * gt).sum().backward()
    scene = oracle.Scene(ref_sp, scale=sc, opacity=op, beta=0.25)
    ref_img = oracle.trace(scene, cli)["rgba"]
    err = np.abs(img.detach().cpu().numpy().reshape(-1, 4) - ref_img)
    assert err.max() <= 2e-3 and err.mean() <= 1e-4
    rr, ro, rs = oracle.trace_backward(scene, cli, g.astype(np.float64))
    assert_elementwise(col.grad.cpu().numpy(), rr, "autograd rgba")
    assert_elementwise(opt.grad.cpu().numpy(), ro, "autograd opacity")
    assert_elementwise(sct.grad.cpu().numpy(), rs, "autograd scale", atol=ATOL_SCALE)


# ---------------------------------------------------------------------------------------------
# the differentiation workload's size: 512^2 server image, 262,144 splats, 512^2 views
# ---------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def diff_scene(wrs):
    W = synth.DIFF
    srv = W.server_cam()
    rgba, depth = oracle.raycast(W.volume(), synth.tf_ramp(), srv)
    rgba = rgba.astype(np.float32)
    ref_sp = oracle.unproject(rgba, depth, srv)
    n = ref_sp.n
    rng = np.random.default_rng(55)
    sc = rng.uniform(0.8, 1.6, n).astype(np.float32)  # radius scales near their start value 1.0
    op = np.ones(n, np.float32)
    sp = wrs.unproject(_cuda(rgba), _cuda(depth), srv)
    assert sp.count() == n
    return sp, ref_sp, sc, op, W.client_poses()


@pytest.mark.parametrize("sched,k", [(2, 4), (0, 2)])
def test_backward_diff_workload_one_view(wrs, diff_scene, sched, k):
    sp, ref_sp, sc, op, cams = diff_scene
    n = ref_sp.n
    cli = cams[3]
    bvh, srt = wrs.build_lbvh(sp, 1, radius_scale=_cuda(sc))
    g = np.random.default_rng(7).normal(size=(cli.height * cli.width, 4)).astype(np.float32)
    params = wrs.TraceParams(edge_softness=0.25, k_chunk=k, schedule=sched, width=4)
    st = wrs.new_status()
    gr, go, gs = wrs.trace_backward(bvh, srt, cli, _cuda(g.reshape(cli.height, cli.width, 4)),
                                    params, opacity=_cuda(op), radius_scale=_cuda(sc), status=st)
    wrs.check_status(st)
    scene = oracle.Scene(ref_sp, scale=sc, opacity=op, beta=0.25)
    rr, ro, rs = oracle.trace_backward(scene, cli, g.astype(np.float64))
    assert np.count_nonzero(rs) > n // 10  # splats some ray meets inside the soft-edge band
    what = f"diff 512^2 schedule={sched} K={k}"
    assert_elementwise(gr.cpu().numpy()[:n], rr, f"{what} rgba")
    assert_elementwise(go.cpu().numpy()[:n], ro, f"{what} opacity")
    assert_elementwise(gs.cpu().numpy()[:n], rs, f"{what} scale", atol=ATOL_SCALE)


@pytest.fixture(scope="module")
def diff_eight_views(diff_scene):
    """Random upstream gradients of the 8 views and the sum of the 8 oracle adjoints (computed once
    for the tests below)."""
    sp, ref_sp, sc, op, cams = diff_scene
    n = ref_sp.n
    V = len(cams)
    h, w = cams[0].height, cams[0].width
    g = np.random.default_rng(8).normal(size=(V, h * w, 4)).astype(np.float32)
    scene = oracle.Scene(ref_sp, scale=sc, opacity=op, beta=0.25)
    rr = np.zeros((n, 4))
    ro = np.zeros(n)
    rs = np.zeros(n)
    for v, cam in enumerate(cams):
        a, b, c = oracle.trace_backward(scene, cam, g[v].astype(np.float64))
        rr += a
        ro += b
        rs += c
    return g.reshape(V, h, w, 4), rr, ro, rs


# the packet launch and the per-pixel launch the bench's tuner picks (K 4, 8 resident blocks)
@pytest.mark.parametrize("sched", [2, 0])
def test_backward_diff_workload_eight_views_one_launch(wrs, diff_scene, diff_eight_views, sched):
    """All 8 views of the differentiation workload in one backward launch: the accumulated
    gradient against the sum of the 8 oracle adjoints."""
    sp, ref_sp, sc, op, cams = diff_scene
    g, rr, ro, rs = diff_eight_views
    n = ref_sp.n
    bvh, srt = wrs.build_lbvh(sp, 1, radius_scale=_cuda(sc))
    params = wrs.TraceParams(edge_softness=0.25, k_chunk=4, schedule=sched, width=4)
    st = wrs.new_status()
    gr, go, gs = wrs.trace_backward_views(bvh, srt, cams, _cuda(g), params,
                                          opacity=_cuda(op), radius_scale=_cuda(sc), status=st)
    wrs.check_status(st)
    what = f"diff 8 views schedule={sched}"
    assert_elementwise(gr.cpu().numpy()[:n], rr, f"{what} rgba")
    assert_elementwise(go.cpu().numpy()[:n], ro, f"{what} opacity")
    assert_elementwise(gs.cpu().numpy()[:n], rs, f"{what} scale", atol=ATOL_SCALE)


# ---------------------------------------------------------------------------------------------
# GPU gradient against central finite differences of the GPU forward
# ---------------------------------------------------------------------------------------------
def test_gpu_gradient_matches_central_differences(wrs):
    """64x64 server image without holes (4,096 splats), a client 10 degrees away, beta = 0.25,
    loss L = sum(g * image) evaluated in binary64 on the host.  For 48 splats that the view
    reaches: red and alpha of the colour, opacity and radius scale, each against
    (L(p + h) - L(p - h)) / 2h with h = 1e-3.  Parameters whose +-h changes any hit list (the
    oracle's binary32 hit lists, the GPU's own) are skipped and counted."""
    rgba, depth, srv, cli, ref_sp, op, sc, g = _bwd_instance(64, 64, 11, hole_frac=0.0)
    n = ref_sp.n
    assert n == 4096
    op = np.minimum(op, 0.95).astype(np.float32)
    h = 1e-3
    sp = wrs.unproject(_cuda(rgba), _cuda(depth), srv)
    params = wrs.TraceParams(edge_softness=0.25)
    gt = g.astype(np.float64)

    def render(col, opa, scl):
        img = wrs.render(sp, cli, _cuda(col), _cuda(opa), _cuda(scl), params)
        return img.detach().cpu().numpy().astype(np.float64).reshape(-1, 4)

    def loss(col, opa, scl):
        return float(np.sum(gt * render(col, opa, scl)))

    col = ref_sp.rgba.copy()
    col_t = torch.tensor(col, device="cuda", requires_grad=True)
    op_t = torch.tensor(op, device="cuda", requires_grad=True)
    sc_t = torch.tensor(sc, device="cuda", requires_grad=True)
    img = wrs.render(sp, cli, col_t, op_t, sc_t, params)
    (img * _cuda(g.reshape(cli.height, cli.width, 4))).sum().backward()
    grads = {"red": col_t.grad.cpu().numpy()[:, 0], "alpha": col_t.grad.cpu().numpy()[:, 3],
             "opacity": op_t.grad.cpu().numpy(), "scale": sc_t.grad.cpu().numpy()}
    reached = np.flatnonzero(np.abs(grads["opacity"]) > 0)
    pick = np.random.default_rng(3).choice(reached, 48, replace=False)

    def hashes(scl):
        return oracle.trace(oracle.Scene(ref_sp, scale=scl, opacity=op, beta=0.25), cli)["hash"]

    base_hash = hashes(sc)
    skipped = checked = 0
    for name in ("red", "alpha", "opacity", "scale"):
        gmax = np.abs(grads[name]).max()
        for i in pick:
            args_p = [col.copy(), op.copy(), sc.copy()]
            args_m = [col.copy(), op.copy(), sc.copy()]
            if name == "red":
                args_p[0][i, 0] += h
                args_m[0][i, 0] -= h
            elif name == "alpha":
                args_p[0][i, 3] += h
                args_m[0][i, 3] -= h
            elif name == "opacity":
                args_p[1][i] += h
                args_m[1][i] -= h
            else:
                args_p[2][i] += h
                args_m[2][i] -= h
                if not (np.array_equal(hashes(args_p[2]), base_hash)
                        and np.array_equal(hashes(args_m[2]), base_hash)):
                    skipped += 1
                    continue
            fd = (loss(*args_p) - loss(*args_m)) / (2 * h)
            got = float(grads[name][i])
            assert abs(fd - got) <= 1e-2 * abs(fd) + 2e-3 * gmax, (name, int(i), got, fd)
            checked += 1
    print(f"finite differences: {checked} parameters checked, {skipped} skipped (hit list changes)")
    assert checked >= 4 * 48 - 24


@pytest.mark.parametrize("sched", [2, 0])
def test_recorded_adjoint_diff_workload_eight_views(wrs, diff_scene, diff_eight_views, sched):
    """The 8 views of the differentiation workload with recorded hit lists (the forward pass
    records, the adjoint runs without traversal): the accumulated gradient against the sum of the
    8 oracle adjoints, element by element."""
    sp, ref_sp, sc, op, cams = diff_scene
    g, rr, ro, rs = diff_eight_views
    n = ref_sp.n
    bvh, srt = wrs.build_lbvh(sp, 1, radius_scale=_cuda(sc))
    params = wrs.TraceParams(edge_softness=0.25, k_chunk=4, schedule=sched, width=4)
    st = wrs.new_status()
    _, lists = wrs.trace_views_record(bvh, srt, cams, params, 16, opacity=_cuda(op), status=st)
    over = int((lists.count > 16).sum())
    gr, go, gs = wrs.trace_backward_views_recorded(bvh, srt, cams, lists, _cuda(g), params,
                                                   opacity=_cuda(op), radius_scale=_cuda(sc),
                                                   status=st)
    wrs.check_status(st)
    print(f"rays over the list capacity (re-traversed): {over}")
    what = f"recorded 8 views schedule={sched}"
    assert_elementwise(gr.cpu().numpy()[:n], rr, f"{what} rgba")
    assert_elementwise(go.cpu().numpy()[:n], ro, f"{what} opacity")
    assert_elementwise(gs.cpu().numpy()[:n], rs, f"{what} scale", atol=ATOL_SCALE)
