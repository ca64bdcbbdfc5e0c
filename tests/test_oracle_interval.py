"""Oracle pins: samples smeared along their viewing ray over a depth interval, as chains of touching
spheres (future work, §6; reading: spec S3b).

Expected values come from the geometry of the server rays (distances along each ray, the footprint
closed form), the composition law of n equal opacities, and the server view, which a chain must
composite back to the pixel's own colour.
"""
import math

import numpy as np

import synth


def _image(W, H, seed, interval):
    rgba, depth = synth.synthetic_server_image(W, H, seed)
    hi = depth.copy()
    fin = np.isfinite(depth)
    hi[fin] = depth[fin] * np.float32(1.0 + interval)
    return rgba, depth, hi.astype(np.float32)


def test_zero_interval_is_the_plain_unprojection(orc):
    W, H = 37, 29
    rgba, depth, _ = _image(W, H, 3, 0.0)
    cam = synth.server_camera(1.4, 30.0, W, H)
    a = orc.unproject(rgba, depth, cam)
    b = orc.unproject_interval(rgba, depth, depth, cam, max_chain=8)
    assert np.array_equal(a.pos_r.view(np.uint32), b.pos_r.view(np.uint32))
    assert np.array_equal(a.rgba.view(np.uint32), b.rgba.view(np.uint32))
    assert np.array_equal(b.id, a.id * 8)


def test_chain_geometry_and_opacity(orc):
    """Along each pixel's ray, n = ceil(L / 2 r0) spheres (capped) at t_lo + (2k+1) L / 2n, so
    neighbours touch or overlap; their opacities a' compose to the pixel's a."""
    W, H = 24, 18
    rgba, depth, hi = _image(W, H, 4, 0.05)
    cam = synth.server_camera(1.4, 30.0, W, H)
    sp = orc.unproject_interval(rgba, depth, hi, cam, max_chain=16)
    eye = np.array(cam.eye, np.float64)
    pitch = 2 * cam.tan_half_fovy / H
    pix = sp.id // 16
    k = sp.id % 16
    for i in np.unique(pix)[::5]:
        sel = np.flatnonzero(pix == i)
        t_lo, t_hi = float(depth.reshape(-1)[i]), float(hi.reshape(-1)[i])
        L = t_hi - t_lo
        x, y = i % W, i // W
        # the footprint radius at the interval's middle (S3 closed form, binary64)
        u = ((2 * x + 1) / W - 1) * cam.tan_half_fovy * W / H
        v = (1 - (2 * y + 1) / H) * cam.tan_half_fovy
        dz = 1 / math.sqrt(1 + u * u + v * v)
        r0 = (t_lo + L / 2) * dz * pitch * math.sqrt(0.5)
        n = min(max(math.ceil(L / (2 * r0) - 1e-6), 1), 16)
        assert len(sel) == n and np.array_equal(k[sel], np.arange(n))
        dist = np.linalg.norm(sp.pos_r[sel, :3].astype(np.float64) - eye, axis=1)
        want = t_lo + (2 * np.arange(n) + 1) * L / (2 * n)
        assert np.allclose(dist, want, rtol=0, atol=2e-6 * (1 + t_hi))
        assert L / n <= 2 * r0 * (1 + 1e-5)  # neighbours touch or overlap
        a = float(rgba.reshape(-1, 4)[i, 3])
        ap = sp.rgba[sel, 3].astype(np.float64)
        assert np.allclose(ap, ap[0])
        assert abs(1 - (1 - ap[0]) ** n - a) < 1e-6
        # premultiplied colour scaled like the alpha
        assert np.allclose(sp.rgba[sel[0], :3] / ap[0], rgba.reshape(-1, 4)[i, :3] / a, rtol=1e-5)


def test_chain_is_capped(orc):
    W, H = 12, 10
    rgba, depth, hi = _image(W, H, 5, 0.5)  # long intervals
    cam = synth.server_camera(1.4, 30.0, W, H)
    sp = orc.unproject_interval(rgba, depth, hi, cam, max_chain=3)
    counts = np.bincount(sp.id // 3)
    assert counts.max() == 3 and len(np.unique(sp.id)) == sp.n


def test_server_view_composites_back_to_the_image(orc):
    """Seen from the server camera each ray passes through its own chain only (short intervals:
    neighbouring chains stay off the ray), and n spheres of opacity a' with colour c a'/a
    composite to c: the server image, up to the records' binary32 rounding."""
    W, H = 40, 30
    rgba, depth, hi = _image(W, H, 6, 0.03)
    cam = synth.server_camera(1.4, 30.0, W, H)
    sp = orc.unproject_interval(rgba, depth, hi, cam, max_chain=8)
    assert sp.n >= 2 * np.isfinite(depth).sum()  # every pixel became a chain of two or more
    img = orc.trace(orc.Scene(sp), cam)["rgba"].reshape(H, W, 4)
    assert np.abs(img - rgba.astype(np.float64)).max() < 2e-6
