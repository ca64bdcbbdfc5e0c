"""GPU parity of the 64-bit quantised splat word and 32-bit colour (§4.1, §6; layout: spec S11)
through the C ABI: every word, colour and decoded record bitwise against the oracle's codec."""
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


BOX = ((0.0, 0.0, 0.0), (1.0, 1.0, 1.0))


def _frame(W, H, seed):
    rgba, depth = synth.synthetic_server_image(W, H, seed)
    return rgba, depth, synth.server_camera(1.4, 30.0, W, H)


def _check_stream(enc, word, color):
    k = enc.count()
    assert k == len(word)
    assert np.array_equal(enc.word[:k].cpu().numpy().view(np.uint64), word)
    assert np.array_equal(enc.color[:k].cpu().numpy().view(np.uint32), color)


@pytest.mark.parametrize("W,H,mode", [(61, 47, 0), (128, 96, 1), (1920, 1080, 0)])
def test_unproject_encode_bitwise(wrs, W, H, mode):
    rgba, depth, cam = _frame(W, H, 31 + W)
    diag = 3 ** 0.5 / 256
    ref = oracle.unproject(rgba, depth, cam, mode, diag)
    r_max = float(ref.pos_r[:, 3].max()) * 0.75  # some radii above the bound: clamped codes
    codec = wrs.make_codec(*BOX, r_max)
    word, color = oracle.encode(ref, *BOX, r_max)
    enc = wrs.unproject_encode(_cuda(rgba), _cuda(depth), cam, codec, mode, diag)
    _check_stream(enc, word, color)
    # the separate encode of the float records gives the same stream
    sp = wrs.unproject(_cuda(rgba), _cuda(depth), cam, mode, diag)
    _check_stream(wrs.encode_splats(sp, codec), word, color)
    # decode: float records bitwise, ids = stream index
    dec = wrs.decode_splats(enc, codec)
    want = oracle.decode(word, color, *BOX, r_max)
    pos, col, ids = (t.cpu().numpy() for t in dec.view())
    assert np.array_equal(pos.view(np.uint32), want.pos_r.view(np.uint32))
    assert np.array_equal(col.view(np.uint32), want.rgba.view(np.uint32))
    assert np.array_equal(ids.view(np.uint32), np.arange(len(word), dtype=np.uint32))


def test_odd_box_clamps_like_the_oracle(wrs):
    """A box that cuts through the cloud: out-of-box points clamp to the border cells."""
    rgba, depth, cam = _frame(80, 60, 41)
    ref = oracle.unproject(rgba, depth, cam)
    lo, hi = (0.3, 0.25, 0.4), (0.7, 0.6, 0.55)
    r_max = 0.002
    word, color = oracle.encode(ref, lo, hi, r_max)
    enc = wrs.unproject_encode(_cuda(rgba), _cuda(depth), cam, wrs.make_codec(lo, hi, r_max))
    _check_stream(enc, word, color)


def test_decoded_trace_matches_oracle(wrs):
    """Decode -> LBVH -> trace on the GPU against the oracle's trace of its decoded splats."""
    rgba, depth, cam = _frame(128, 96, 43)
    ref = oracle.unproject(rgba, depth, cam)
    r_max = float(ref.pos_r[:, 3].max())
    word, color = oracle.encode(ref, *BOX, r_max)
    codec = wrs.make_codec(*BOX, r_max)
    dec = wrs.decode_splats(wrs.unproject_encode(_cuda(rgba), _cuda(depth), cam, codec), codec)
    bvh, srt = wrs.build_lbvh(dec, 1)
    cli = synth.orbit(cam, (0, 1, 0), 6.0, 160, 120)
    img = wrs.trace(bvh, srt, cli, wrs.TraceParams(width=4))
    want = oracle.trace(oracle.Scene(oracle.decode(word, color, *BOX, r_max)), cli)
    err = np.abs(img.cpu().numpy().reshape(-1, 4).astype(np.float64) - want["rgba"])
    assert err.max() <= 1e-5 and err.mean() <= 1e-4


def test_empty_stream_and_bad_codec(wrs):
    cam = synth.server_camera(1.4, 30.0, 16, 8)
    holes = np.full((8, 16), np.inf, np.float32)
    enc = wrs.unproject_encode(_cuda(np.zeros((8, 16, 4), np.float32)), _cuda(holes), cam,
                               wrs.make_codec(*BOX, 0.01))
    assert enc.count() == 0
    assert wrs.decode_splats(enc, wrs.make_codec(*BOX, 0.01)).count() == 0
    for bad in (wrs.make_codec((0, 0, 0), (1, 0, 1), 0.01), wrs.make_codec(*BOX, 0.0),
                wrs.make_codec((0, 0, 0), (1, 1, float("inf")), 0.01)):
        with pytest.raises(wrs.WrsError):
            wrs.unproject_encode(_cuda(np.zeros((8, 16, 4), np.float32)), _cuda(holes), cam, bad)
