"""Oracle pins: the earlier point-splat warping the paper compares against (§2, §5, Fig. 3; reading:
spec S10) and the PSNR used to restate Fig. 3 numerically.

Expected values come from the camera model run backwards (points placed inside a chosen pixel's
cone), the identity warp (server view = client view reproduces the server image), counting covered
pixels, and depth-order cases built by hand.
"""
import math

import numpy as np

import synth


def _splats(orc, pts, cols):
    pts = np.asarray(pts, np.float32).reshape(-1, 3)
    pos_r = np.concatenate([pts, np.full((len(pts), 1), 0.01, np.float32)], axis=1)
    return orc.Splats(pos_r, np.asarray(cols, np.float32).reshape(-1, 4),
                      np.arange(len(pts), dtype=np.uint32))


def _point_in_pixel(cam, x, y, t, dx=0.0, dy=0.0):
    """A point at distance-along-axis t inside the cone of pixel (x, y), offset (dx, dy) pixels
    from its centre (the camera model of S1 run in binary64)."""
    W, H = cam.width, cam.height
    u = ((2 * (x + dx) + 1) / W - 1) * cam.tan_half_fovy * W / H
    v = (1 - (2 * (y + dy) + 1) / H) * cam.tan_half_fovy
    e = np.array(cam.fwd, np.float64) + u * np.array(cam.right, np.float64) + v * np.array(cam.up, np.float64)
    return np.array(cam.eye, np.float64) + t * e


def test_identity_warp_reproduces_the_server_image(orc):
    """Client camera = server camera, size 1: every sample lands on its own pixel."""
    W, H = 57, 43
    rgba, depth = synth.synthetic_server_image(W, H, 5)
    cam = synth.server_camera(1.4, 30.0, W, H)
    sp = orc.unproject(rgba, depth, cam)
    out, idx = orc.point_splat(sp, cam, 1)
    keep = (np.isfinite(depth) & (depth >= 0) & (rgba[..., 3] > 0)).reshape(-1)
    assert np.array_equal(idx.reshape(-1)[keep], np.arange(sp.n))
    assert np.all(idx.reshape(-1)[~keep] == -1)
    assert np.array_equal(out.reshape(-1, 4)[keep].view(np.uint32), rgba.reshape(-1, 4)[keep].view(np.uint32))
    assert not out.reshape(-1, 4)[~keep].any()


def test_points_land_in_the_pixel_whose_cone_holds_them(orc):
    cam = synth.look_at((0.3, 0.8, 2.1), (0.5, 0.5, 0.5), (0, 1, 0), 40.0, 64, 48)
    rng = np.random.default_rng(3)
    for _ in range(60):
        x, y = int(rng.integers(0, 64)), int(rng.integers(0, 48))
        dx, dy = rng.uniform(-0.45, 0.45, size=2)
        p = _point_in_pixel(cam, x, y, rng.uniform(0.5, 3.0), dx, dy)
        out, idx = orc.point_splat(_splats(orc, p, [1, 1, 1, 1]), cam, 1)
        assert np.argwhere(idx == 0).tolist() == [[y, x]]


def test_size_covers_a_square_of_that_many_pixels(orc):
    cam = synth.look_at((0.5, 0.5, 2.0), (0.5, 0.5, 0.5), (0, 1, 0), 30.0, 80, 60)
    for s in (1, 2, 3, 4, 7):
        for dx, dy in ((0.0, 0.0), (0.3, -0.2), (-0.49, 0.49)):
            p = _point_in_pixel(cam, 40, 30, 1.5, dx, dy)
            _, idx = orc.point_splat(_splats(orc, p, [1, 0, 0, 1]), cam, s)
            ys, xs = np.nonzero(idx == 0)
            assert len(xs) == s * s
            assert xs.max() - xs.min() == s - 1 and ys.max() - ys.min() == s - 1
            # the square is centred on the projected point: its centre is within half a pixel
            assert abs((xs.min() + xs.max()) / 2 - (40 + dx)) <= 0.5 + 1e-9
            assert abs((ys.min() + ys.max()) / 2 - (30 + dy)) <= 0.5 + 1e-9
            if s % 2 == 1:
                assert idx[30, 40] == 0


def test_depth_test_keeps_the_nearer_point_in_either_order(orc):
    cam = synth.look_at((0.5, 0.5, 2.0), (0.5, 0.5, 0.5), (0, 1, 0), 30.0, 32, 32)
    near, far = _point_in_pixel(cam, 10, 12, 1.0), _point_in_pixel(cam, 10, 12, 1.6)
    red, blue = [0.5, 0, 0, 0.5], [0, 0, 0.9, 0.9]
    for pts, cols, want in (([near, far], [red, blue], 0), ([far, near], [blue, red], 1)):
        out, idx = orc.point_splat(_splats(orc, pts, cols), cam, 3)
        assert idx[12, 10] == want
        assert np.array_equal(out[12, 10], np.float32(red))
    # coincident points: the lower index wins
    out, idx = orc.point_splat(_splats(orc, [near, near], [red, blue]), cam, 2)
    assert set(np.unique(idx)) == {-1, 0}


def test_points_behind_the_eye_and_far_off_screen_draw_nothing(orc):
    cam = synth.look_at((0.5, 0.5, 2.0), (0.5, 0.5, 0.5), (0, 1, 0), 30.0, 32, 24)
    eye, fwd = np.array(cam.eye, np.float64), np.array(cam.fwd, np.float64)
    right = np.array(cam.right, np.float64)
    pts = [eye - 0.5 * fwd, eye, eye + 1.0 * fwd + 5.0 * right]
    out, idx = orc.point_splat(_splats(orc, pts, [[1, 1, 1, 1]] * 3), cam, 5)
    assert np.all(idx == -1) and not out.any()


def test_border_points_are_clipped(orc):
    cam = synth.look_at((0.5, 0.5, 2.0), (0.5, 0.5, 0.5), (0, 1, 0), 30.0, 32, 24)
    p = _point_in_pixel(cam, 0, 23, 1.2)
    _, idx = orc.point_splat(_splats(orc, p, [1, 1, 1, 1]), cam, 5)
    assert int((idx == 0).sum()) == 3 * 3  # a 5 x 5 square centred on the corner pixel, clipped


def test_psnr_closed_forms(orc):
    a = np.zeros((4, 4, 4))
    assert orc.psnr(a, a) == math.inf
    assert abs(orc.psnr(a + 0.1, a) - 20.0) < 1e-9
    b = a.copy()
    b[0, 0, 0] = 1.0  # MSE = 1/64
    assert abs(orc.psnr(b, a) - 10 * math.log10(64)) < 1e-9
