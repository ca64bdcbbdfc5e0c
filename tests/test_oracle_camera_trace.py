"""Oracle pins: camera (Eq. 1), ray-sphere test (§4 'real quadrics'), compositing (spec S6).

Every expectation here comes from geometry or algebra computed independently of the oracle's
own formulas: a forward projection instead of ray generation, a cone angle instead of the
quadratic, closed-form composites of two layers, brute-force nearest hits in binary64.
"""
import math

import numpy as np
import pytest

import synth


def _cam(eye=(0.5, 0.5, 3.0), target=(0.5, 0.5, 0.5), up=(0, 1, 0), fovy=40.0, W=64, H=48):
    return synth.look_at(eye, target, up, fovy, W, H)


def _project(cam, P):
    """Textbook pinhole projection of a world point to continuous pixel coordinates."""
    eye = np.array(cam.eye, np.float64)
    R, U, F = (np.array(v, np.float64) for v in (cam.right, cam.up, cam.fwd))
    q = np.asarray(P, np.float64) - eye
    z = q @ F
    aspect = cam.width / cam.height
    xn = (q @ R) / z / (cam.tan_half_fovy * aspect)
    yn = (q @ U) / z / cam.tan_half_fovy
    return (xn + 1) / 2 * cam.width - 0.5, (1 - yn) / 2 * cam.height - 0.5


def _splats(orc, pos, r, rgba, ids=None):
    pos = np.asarray(pos, np.float32).reshape(-1, 3)
    n = pos.shape[0]
    pos_r = np.zeros((n, 4), np.float32)
    pos_r[:, :3] = pos
    pos_r[:, 3] = r
    ids = np.arange(n, dtype=np.uint32) if ids is None else np.asarray(ids, np.uint32)
    return orc.Splats(pos_r, np.asarray(rgba, np.float32).reshape(n, 4), ids)


def test_ray_unit_length_and_origin(orc):
    cam = _cam()
    for x, y in [(0, 0), (63, 47), (31, 20), (10, 40)]:
        o, d = orc.primary_ray(cam, x, y)
        assert np.array_equal(o, np.array(cam.eye, np.float32))
        assert abs(float(np.linalg.norm(d.astype(np.float64))) - 1.0) < 1e-6


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ray_passes_through_projected_point(orc, seed):
    """A world point projected with the textbook formula lies on (near) its pixel's ray: pins the
    y-down convention, the aspect ratio on x, and the handedness of right/up."""
    rng = np.random.default_rng(seed)
    cam = _cam(eye=(0.3, 0.8, 2.5), target=(0.6, 0.4, 0.5), up=(0.1, 1, 0), W=80, H=50)
    half_pixel = cam.tan_half_fovy / cam.height  # half a pixel's angular size (small angle)
    for _ in range(50):
        P = rng.uniform(0.2, 0.8, 3)
        px, py = _project(cam, P)
        if not (0 <= px < cam.width - 1 and 0 <= py < cam.height - 1):
            continue
        x, y = int(round(px)), int(round(py))
        o, d = orc.primary_ray(cam, x, y)
        q = P - o.astype(np.float64)
        ang = math.acos(min(1.0, float(q @ d) / float(np.linalg.norm(q))))
        assert ang < 2.0 * half_pixel, (x, y, ang)


def test_orientation_signs(orc):
    cam = _cam(W=32, H=32)
    _, d_left = orc.primary_ray(cam, 0, 16)
    _, d_right = orc.primary_ray(cam, 31, 16)
    _, d_top = orc.primary_ray(cam, 16, 0)
    _, d_bot = orc.primary_ray(cam, 16, 31)
    R, U = np.array(cam.right), np.array(cam.up)
    assert d_right @ R > 0 > d_left @ R
    assert d_top @ U > 0 > d_bot @ U


def test_single_sphere_cone_coverage(orc):
    """A sphere of radius r at distance D covers exactly the pixels whose ray is within the cone
    half-angle asin(r/D) of the centre direction; covered pixels show the sphere's RGBA."""
    cam = _cam(eye=(0.5, 0.5, 2.5), fovy=30.0, W=96, H=96)
    c = np.array([0.55, 0.45, 0.5])
    r = 0.12
    rgba = [0.2, 0.3, 0.1, 0.6]
    sc = orc.Scene(_splats(orc, [c], r, [rgba]))
    out = orc.trace(sc, cam, bvh=None)
    D = np.linalg.norm(c - np.array(cam.eye, np.float64))
    half = math.asin(r / D)
    cover = out["nhits"].reshape(96, 96) > 0
    n_checked = 0
    for y in range(96):
        for x in range(96):
            o, d = orc.primary_ray(cam, x, y)
            q = c - o.astype(np.float64)
            ang = math.acos(min(1.0, float(q @ d.astype(np.float64)) / np.linalg.norm(q)))
            if abs(ang - half) < 1e-5:
                continue  # boundary band: binary32 decides
            n_checked += 1
            assert cover[y, x] == (ang < half), (x, y)
    assert n_checked > 9000
    px = out["rgba"].reshape(96, 96, 4)[cover]
    assert np.abs(px - np.array(rgba, np.float32)).max() < 1e-12
    assert np.all(out["rgba"].reshape(96, 96, 4)[~cover] == 0)
    assert cover.sum() > 100


def test_two_layers_closed_form_and_order(orc):
    """Two spheres on the view axis: front-to-back 'over' c1 + (1-a1) c2, alpha 1-(1-a1)(1-a2);
    swapping depths swaps the order; H = 1 shows only the nearest sphere."""
    cam = _cam(eye=(0.5, 0.5, 3.0), W=33, H=33)
    near, far = [0.5, 0.5, 1.0], [0.5, 0.5, 0.0]
    c1 = np.array([0.1, 0.2, 0.3, 0.4])
    c2 = np.array([0.5, 0.1, 0.2, 0.7])
    sp = _splats(orc, [near, far], 0.3, [c1, c2])
    pix = np.array([16 * 33 + 16])
    o = orc.trace(orc.Scene(sp), cam, pixels=pix, bvh=None)["rgba"][0]
    c1f, c2f = c1.astype(np.float32).astype(np.float64), c2.astype(np.float32).astype(np.float64)
    exp_rgb = c1f[:3] + (1 - c1f[3]) * c2f[:3]
    exp_a = 1 - (1 - c1f[3]) * (1 - c2f[3])
    assert np.allclose(o[:3], exp_rgb, atol=1e-12) and abs(o[3] - exp_a) < 1e-12
    sp2 = _splats(orc, [far, near], 0.3, [c1, c2])
    o2 = orc.trace(orc.Scene(sp2), cam, pixels=pix, bvh=None)["rgba"][0]
    assert np.allclose(o2[:3], c2f[:3] + (1 - c2f[3]) * c1f[:3], atol=1e-12)
    o3 = orc.trace(orc.Scene(sp, max_hits=1), cam, pixels=pix, bvh=None)["rgba"][0]
    assert np.allclose(o3, c1f, atol=1e-12)


def test_origin_inside_ties_broken_by_id(orc):
    """Spheres that contain the eye have key 0; equal keys are composited in id order."""
    cam = _cam(eye=(0.5, 0.5, 0.5), target=(0.5, 0.5, 0.0), W=8, H=8)
    ca = np.array([0.9, 0.0, 0.0, 0.5])
    cb = np.array([0.0, 0.0, 0.9, 0.5])
    sp = _splats(orc, [[0.5, 0.5, 0.5], [0.52, 0.5, 0.5]], 1.0, [ca, cb], ids=[7, 3])
    o = orc.trace(orc.Scene(sp), cam, bvh=None)["rgba"]
    caf, cbf = ca.astype(np.float32).astype(np.float64), cb.astype(np.float32).astype(np.float64)
    exp = cbf[:3] + (1 - cbf[3]) * caf[:3]  # id 3 first
    assert np.allclose(o[:, :3], exp, atol=1e-12)


def test_sphere_behind_camera_is_missed(orc):
    cam = _cam(eye=(0.5, 0.5, 1.0), target=(0.5, 0.5, 0.0), W=8, H=8)
    sp = _splats(orc, [[0.5, 0.5, 2.0]], 0.2, [[1, 1, 1, 1]])
    assert orc.trace(orc.Scene(sp), cam, bvh=None)["nhits"].sum() == 0


def _random_scene(orc, n, seed, alpha_lo=0.05):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.2, 0.8, (n, 3))
    r = rng.uniform(0.005, 0.04, n)
    a = rng.uniform(alpha_lo, 1.0, n)
    rgb = rng.uniform(0, 1, (n, 3)) * a[:, None]
    sp = _splats(orc, pos, 0, np.concatenate([rgb, a[:, None]], 1), ids=rng.permutation(n) + 10)
    sp.pos_r[:, 3] = r
    return sp


def test_nearest_hit_matches_binary64_brute_force(orc):
    """H = 1 shows the sphere with the smallest entry distance (spec S5), found here by an
    independent binary64 brute force over all spheres; pixels with a near-tie are skipped."""
    sp = _random_scene(orc, 300, 3)
    cam = _cam(eye=(0.4, 0.6, 2.2), W=40, H=40)
    out = orc.trace(orc.Scene(sp, max_hits=1), cam, bvh=None)["rgba"]
    c = sp.pos_r[:, :3].astype(np.float64)
    r = sp.pos_r[:, 3].astype(np.float64)
    checked = 0
    for p in range(40 * 40):
        o, d = orc.primary_ray(cam, p % 40, p // 40)
        o, d = o.astype(np.float64), d.astype(np.float64) / np.linalg.norm(d.astype(np.float64))
        oc = c - o
        b = oc @ d
        dist2 = np.sum((oc - b[:, None] * d) ** 2, axis=1)
        hit = dist2 < r * r
        if not hit.any():
            assert np.all(out[p] == 0)
            continue
        entry = b[hit] - np.sqrt(r[hit] ** 2 - dist2[hit])
        order = np.argsort(entry)
        if len(order) > 1 and entry[order[1]] - entry[order[0]] < 1e-6:
            continue
        if np.min(np.abs(dist2[hit] - r[hit] ** 2)) < 1e-9:
            continue
        k = np.flatnonzero(hit)[order[0]]
        assert np.allclose(out[p], sp.rgba[k].astype(np.float64), atol=1e-12), p
        checked += 1
    assert checked > 300


@pytest.mark.parametrize("seed", [4, 5])
def test_bvh_equals_brute_force_bitwise(orc, seed):
    sp = _random_scene(orc, 2000, seed)
    cam = _cam(eye=(0.9, 0.3, 2.0), W=48, H=40)
    for H in (0, 1, 3):
        sc = orc.Scene(sp, max_hits=H)
        a = orc.trace(sc, cam, bvh=None)
        for leaf in (1, 4, 16):
            b = orc.trace(sc, cam, bvh=orc.BVH(sc, leaf=leaf))
            assert np.array_equal(a["rgba"], b["rgba"])
            assert np.array_equal(a["hash"], b["hash"])


def test_permutation_invariance_bitwise(orc):
    sp = _random_scene(orc, 1500, 6)
    cam = _cam(eye=(0.2, 0.5, 2.4), W=40, H=40)
    perm = np.random.default_rng(1).permutation(sp.n)
    sp2 = orc.Splats(sp.pos_r[perm], sp.rgba[perm], sp.id[perm])
    a = orc.trace(orc.Scene(sp), cam)
    b = orc.trace(orc.Scene(sp2), cam)
    assert np.array_equal(a["rgba"], b["rgba"])


def test_pixel_subset_equals_full_image(orc):
    sp = _random_scene(orc, 500, 7)
    cam = _cam(W=30, H=20)
    full = orc.trace(orc.Scene(sp), cam)
    pix = np.array([0, 5, 599, 311, 42])
    sub = orc.trace(orc.Scene(sp), cam, pixels=pix)
    assert np.array_equal(full["rgba"][pix], sub["rgba"])


def test_t_stop_truncation_closed_form(orc):
    """k identical layers of alpha a on the axis: compositing stops once T <= 1e-5, so exactly
    ceil(log(1e-5) / log(1 - a)) layers are used."""
    a = 0.5
    k = 30
    cam = _cam(eye=(0.5, 0.5, 5.0), W=9, H=9)
    pos = [[0.5, 0.5, 1.0 - 0.05 * i] for i in range(k)]
    sp = _splats(orc, pos, 0.02, [[a * 0.5, a * 0.2, a * 0.1, a]] * k)
    out = orc.trace(orc.Scene(sp), cam, pixels=np.array([4 * 9 + 4]), bvh=None)
    used = math.ceil(math.log(1e-5) / math.log(1 - a))
    assert out["nused"][0] == used and out["nhits"][0] == k
    assert abs(out["T"][0] - (1 - a) ** used) < 1e-15


def test_max_hits_limits_layers(orc):
    cam = _cam(eye=(0.5, 0.5, 5.0), W=9, H=9)
    pos = [[0.5, 0.5, 1.0 - 0.05 * i] for i in range(5)]
    sp = _splats(orc, pos, 0.02, [[0.1, 0.1, 0.1, 0.2]] * 5)
    for H, n in [(1, 1), (2, 2), (4, 4), (0, 5), (9, 5)]:
        out = orc.trace(orc.Scene(sp, max_hits=H), cam, pixels=np.array([40]), bvh=None)
        assert out["nused"][0] == n
        assert abs(out["rgba"][0, 3] - (1 - 0.8 ** n)) < 1e-7


def test_soft_edge_weight_closed_form(orc):
    """With edge softness beta, a pixel at normalised distance rho from the centre line shows
    alpha = a * W(rho), W = smoothstep((1 - rho) / beta) beyond 1 - beta (spec S6)."""
    cam = _cam(eye=(0.5, 0.5, 3.0), fovy=20.0, W=64, H=1)
    c = np.array([0.5, 0.5, 0.5])
    r, a, beta = 0.2, 0.8, 0.25
    sp = _splats(orc, [c], r, [[0.4, 0.4, 0.4, a]])
    out = orc.trace(orc.Scene(sp, beta=beta), cam, bvh=None)
    for x in range(64):
        o, d = orc.primary_ray(cam, x, 0)
        o, d = o.astype(np.float64), d.astype(np.float64)
        q = c - o
        dist = np.linalg.norm(q - (q @ d) * d)
        rho = dist / r
        if rho >= 1 or abs(rho - 1) < 1e-5:
            continue
        u = min(1.0, (1 - rho) / beta)
        Wv = u * u * (3 - 2 * u)
        assert abs(out["rgba"][x, 3] - a * Wv) < 1e-6, x
        assert abs(out["rgba"][x, 0] - 0.4 * Wv) < 1e-6


def test_empty_scene(orc):
    sp = orc.Splats(np.zeros((0, 4), np.float32), np.zeros((0, 4), np.float32),
                    np.zeros(0, np.uint32))
    out = orc.trace(orc.Scene(sp), _cam(W=4, H=4), bvh=None)
    assert np.all(out["rgba"] == 0) and np.all(out["T"] == 1)
