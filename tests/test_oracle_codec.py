"""Oracle pins: the 64-bit quantised position + radius word and the 32-bit colour the server sends
(§4.1, §6; bit layout: reading of spec S11).

Expected values come from cell centres that are exact in binary32 (so the word can be built by
hand), the quantisation error bounds of a uniform grid, colour values that are exact multiples of
1/255, and the invariance of the traced image to replacing pixel ids by stream indices.
"""
import numpy as np

import synth


def _splats(orc, pos_r, rgba=None):
    pos_r = np.asarray(pos_r, np.float32).reshape(-1, 4)
    n = len(pos_r)
    if rgba is None:
        rgba = np.full((n, 4), 0.5, np.float32)
    return orc.Splats(pos_r, np.asarray(rgba, np.float32).reshape(-1, 4), np.arange(n, dtype=np.uint32))


def test_word_layout_on_exact_cell_centres(orc):
    """Unit box, r_max = 8191 (radius step 1): a point at the centre of cell (qx, qy, qz) with radius
    qr packs to qx | qy << 17 | qz << 34 | qr << 51 and decodes back to itself exactly."""
    rng = np.random.default_rng(1)
    q = rng.integers(0, 131072, size=(200, 3)).astype(np.uint64)
    q[0] = (0, 0, 0)
    q[1] = (131071, 131071, 131071)
    qr = rng.integers(0, 8192, size=200).astype(np.uint64)
    qr[:2] = (0, 8191)
    pts = ((2 * q.astype(np.float64) + 1) / 2 ** 18).astype(np.float32)
    pos_r = np.concatenate([pts, qr.astype(np.float32)[:, None]], axis=1)
    word, _ = orc.encode(_splats(orc, pos_r), (0, 0, 0), (1, 1, 1), 8191.0)
    want = q[:, 0] | (q[:, 1] << np.uint64(17)) | (q[:, 2] << np.uint64(34)) | (qr << np.uint64(51))
    assert np.array_equal(word, want)
    dec = orc.decode(word, np.zeros(200, np.uint32), (0, 0, 0), (1, 1, 1), 8191.0)
    assert np.array_equal(dec.pos_r.view(np.uint32), pos_r.view(np.uint32))


def test_quantisation_error_bounds(orc):
    rng = np.random.default_rng(2)
    lo, hi = np.float32([-0.3, 0.1, 2.0]), np.float32([1.7, 0.6, 2.25])
    n = 5000
    pts = (lo + rng.uniform(0, 1, size=(n, 3)) * (hi - lo)).astype(np.float32)
    r_max = np.float32(0.004)
    r = rng.uniform(0, 1, size=n).astype(np.float32) * r_max
    col = rng.uniform(0, 1, size=(n, 4)).astype(np.float32)
    sp = _splats(orc, np.concatenate([pts, r[:, None]], axis=1), col)
    word, color = orc.encode(sp, lo, hi, r_max)
    dec = orc.decode(word, color, lo, hi, r_max)
    step = (hi.astype(np.float64) - lo) / 2 ** 17
    err = np.abs(dec.pos_r[:, :3].astype(np.float64) - pts)
    # half a cell, plus the binary32 rounding of (p - lo) * inv (at most 2^17 * 2^-23 = 1/64 of a
    # cell, which can move a point next to a cell boundary into the neighbour) and of the decode
    assert np.all(err <= step * (0.5 + 1 / 64) + 1.2e-7 * np.abs(pts))
    assert np.mean(err <= step / 2 + 1.2e-7 * np.abs(pts)) > 0.95
    rd = dec.pos_r[:, 3].astype(np.float64)
    rstep = float(r_max) / 8191
    assert np.all(rd >= r * (1 - 1e-6)) and np.all(rd <= r + rstep * (1 + 1e-5))
    assert np.max(np.abs(dec.rgba.astype(np.float64) - col)) <= 1 / 510 + 1e-7
    assert np.array_equal(dec.id, np.arange(n, dtype=np.uint32))


def test_colour_codes_and_clamping(orc):
    k = np.arange(256, dtype=np.float64)
    col = np.stack([k / 255] * 4, axis=1).astype(np.float32)
    pos_r = np.tile(np.float32([0.5, 0.5, 0.5, 0.001]), (256, 1))
    _, color = orc.encode(_splats(orc, pos_r, col), (0, 0, 0), (1, 1, 1), 0.01)
    assert np.array_equal(color & 255, np.arange(256, dtype=np.uint32))
    assert np.array_equal(color >> 24, np.arange(256, dtype=np.uint32))
    # outside the box, above r_max, negative or not-a-number: clamped into the code range
    pos_r = np.float32([[-1, 2, 0.5, 1.0], [np.nan, 0.5, 0.5, np.nan], [0.5, 0.5, 1.0, -0.1]])
    word, color = orc.encode(_splats(orc, pos_r, [[2, -1, np.nan, 0.5]] * 3), (0, 0, 0), (1, 1, 1), 0.01)
    m = np.uint64(0x1FFFF)
    assert int(word[0] & m) == 0 and int((word[0] >> np.uint64(17)) & m) == 131071
    assert int(word[0] >> np.uint64(51)) == 8191
    assert int(word[1] & m) == 0 and int(word[1] >> np.uint64(51)) == 0
    assert int((word[2] >> np.uint64(34)) & m) == 131071 and int(word[2] >> np.uint64(51)) == 0
    assert int(color[0] & 255) == 255 and int((color[0] >> 8) & 255) == 0
    assert int((color[0] >> 16) & 255) == 0 and int(color[0] >> 24) == 128


def test_stream_ids_keep_the_image(orc):
    """Decoded splats carry stream indices as ids; the compacted stream is in pixel order, so the
    tie order (and the traced image) is the same as with the pixel ids."""
    W, H = 48, 36
    rgba, depth = synth.synthetic_server_image(W, H, 21)
    cam = synth.server_camera(1.4, 30.0, W, H)
    sp = orc.unproject(rgba, depth, cam)
    r_max = float(sp.pos_r[:, 3].max())
    word, color = orc.encode(sp, (0, 0, 0), (1, 1, 1), r_max)
    dec = orc.decode(word, color, (0, 0, 0), (1, 1, 1), r_max)
    with_pixel_ids = orc.Splats(dec.pos_r, dec.rgba, sp.id)
    cli = synth.orbit(cam, (0, 1, 0), 7.0, 40, 30)
    a = orc.trace(orc.Scene(dec), cli)
    b = orc.trace(orc.Scene(with_pixel_ids), cli)
    assert np.array_equal(a["rgba"], b["rgba"]) and np.array_equal(a["nhits"], b["nhits"])
    # and the decoded view stays close to the original one
    c = orc.trace(orc.Scene(sp), cli)
    assert orc.psnr(a["rgba"], c["rgba"]) > 25.0
