"""The packet schedule (one warp-shared traversal of the 4-wide nodes per 8x4 tile) gives the same
images as the per-ray schedules, bitwise, and matches the oracle."""
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


@pytest.mark.parametrize("H,k,block,beta", [(0, 1, 128, 0.0), (0, 4, 256, 0.0), (1, 1, 64, 0.0),
                                            (3, 2, 128, 0.25), (0, 16, 128, 0.0)])
def test_packet_equals_per_pixel_bitwise(wrs, H, k, block, beta):
    """Ragged 133 x 97 client (partial warps at the edges), several k-buffer sizes."""
    rgba, depth = synth.synthetic_server_image(160, 120, 61)
    srv = synth.server_camera(1.4, 30.0, 160, 120)
    cli = synth.orbit(srv, (0.3, 1.0, 0.0), 9.0, 133, 97)
    sp = wrs.unproject(_cuda(rgba), _cuda(depth), srv)
    bvh, srt = wrs.build_lbvh(sp, 1)
    st = wrs.new_status()
    base = wrs.trace(bvh, srt, cli, wrs.TraceParams(max_hits=H, edge_softness=beta, k_chunk=k,
                                                    width=4), status=st)
    pk = wrs.trace(bvh, srt, cli, wrs.TraceParams(max_hits=H, edge_softness=beta, k_chunk=k,
                                                  block=block, schedule=wrs.SCHEDULE_PACKET),
                   status=st)
    wrs.check_status(st)
    assert torch.equal(base, pk)
    ref = oracle.trace(oracle.Scene(oracle.unproject(rgba, depth, srv), max_hits=H, beta=beta), cli)
    err = np.abs(pk.cpu().numpy().reshape(-1, 4).astype(np.float64) - ref["rgba"])
    assert err.max() <= 2e-4 and err.mean() <= 1e-4


def test_packet_large_sampled_and_layers(wrs):
    """1080p / 2 M splats on sampled pixels, and a 40-layer stack that needs many passes."""
    rgba, depth = synth.synthetic_server_image(1920, 1080, 51)
    srv = synth.LARGE.server_cam()
    cli = synth.orbit(srv, (0.6, 0.8, 0.0), 20.0)
    sp = wrs.unproject(_cuda(rgba), _cuda(depth), srv)
    bvh, srt = wrs.build_lbvh(sp, 1)
    st = wrs.new_status()
    a = wrs.trace(bvh, srt, cli, wrs.TraceParams(k_chunk=1, width=4), status=st)
    b = wrs.trace(bvh, srt, cli, wrs.TraceParams(k_chunk=1, schedule=wrs.SCHEDULE_PACKET), status=st)
    wrs.check_status(st)
    assert torch.equal(a, b)
    # 40 stacked translucent layers: every ray gathers far more than K hits over many passes
    W, Hh = 48, 40
    layers = []
    rng = np.random.default_rng(5)
    for L in range(40):
        rgba_l = np.zeros((Hh, W, 4), np.float32)
        rgba_l[..., 3] = 0.08
        rgba_l[..., :3] = rng.uniform(0, 0.08, size=(Hh, W, 3))
        layers.append((rgba_l, np.full((Hh, W), 1.0 + 0.01 * L, np.float32)))
    srv2 = synth.server_camera(1.4, 30.0, W, Hh)
    acc = wrs.SplatBuffers(40 * W * Hh)
    wrs.unproject(_cuda(layers[0][0]), _cuda(layers[0][1]), srv2, out=acc)
    for L in range(1, 40):
        wrs.unproject_append(_cuda(layers[L][0]), _cuda(layers[L][1]), srv2, acc, id_base=L * W * Hh)
    bvh2, srt2 = wrs.build_lbvh(acc, 1)
    cli2 = synth.orbit(srv2, (0, 1, 0), 2.0, 40, 36)
    for k in (1, 2, 16):
        a = wrs.trace(bvh2, srt2, cli2, wrs.TraceParams(k_chunk=k, width=4, t_stop=1e-6), status=st)
        b = wrs.trace(bvh2, srt2, cli2, wrs.TraceParams(k_chunk=k, schedule=wrs.SCHEDULE_PACKET,
                                                        t_stop=1e-6), status=st)
        wrs.check_status(st)
        assert torch.equal(a, b), k
