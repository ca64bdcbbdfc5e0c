"""Oracle pins: unprojection (Eq. 1, §4.1), radius rules (§4.1), compaction (§4.1), the server's
volume ray caster and its first-hit depth heuristic (§4.1, §4.2, Fig. 2).

Expected values come from geometry (distances along rays, cone angles of pixels), closed forms of
compositing through a homogeneous medium, and volumes whose threshold crossing is known.
"""
import json
import math
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _img(H, W, seed):
    return synth.synthetic_server_image(W, H, seed)


def test_compaction_count_order_and_copy(orc):
    rgba, depth = _img(37, 53, 1)
    depth[3, 4] = -1.0          # negative depth: not a sample
    depth[5, 6] = np.nan        # not a number: not a sample
    rgba[7, 8, 3] = 0.0         # zero opacity: radius zero, compacted away
    cam = synth.server_camera(1.4, 30.0, 53, 37)
    sp = orc.unproject(rgba, depth, cam)
    keep = np.isfinite(depth) & (depth >= 0) & (rgba[..., 3] > 0)
    assert sp.n == int(keep.sum())
    assert np.array_equal(sp.id, np.flatnonzero(keep.reshape(-1)).astype(np.uint32))
    assert np.array_equal(sp.rgba.view(np.uint32), rgba.reshape(-1, 4)[keep.reshape(-1)].view(np.uint32))


def test_empty_image_gives_no_splats(orc):
    cam = synth.server_camera(1.4, 30.0, 16, 8)
    sp = orc.unproject(np.zeros((8, 16, 4), np.float32), np.full((8, 16), np.inf, np.float32), cam)
    assert sp.n == 0


def test_unprojected_point_lies_on_its_ray_at_distance_t(orc):
    """Eq. 1: p = o + d t_i.  Checked against the textbook projection of p back to its pixel and
    its Euclidean distance from the eye."""
    W, H = 40, 30
    rgba, depth = _img(H, W, 2)
    cam = synth.look_at((0.2, 0.7, 1.9), (0.5, 0.5, 0.5), (0, 1, 0), 35.0, W, H)
    sp = orc.unproject(rgba, depth, cam)
    eye = np.array(cam.eye, np.float64)
    R, U, F = (np.array(v, np.float64) for v in (cam.right, cam.up, cam.fwd))
    for k in range(0, sp.n, 7):
        p = sp.pos_r[k, :3].astype(np.float64)
        i = int(sp.id[k])
        t = float(depth.reshape(-1)[i])
        assert abs(np.linalg.norm(p - eye) - t) < 2e-6 * (1 + t)
        q = p - eye
        z = q @ F
        px = ((q @ R) / z / (cam.tan_half_fovy * W / H) + 1) / 2 * W - 0.5
        py = (1 - (q @ U) / z / cam.tan_half_fovy) / 2 * H - 0.5
        assert abs(px - i % W) < 1e-3 and abs(py - i // W) < 1e-3


def test_footprint_radius_is_half_pixel_diagonal(orc):
    """Footprint mode: r0 = half the diagonal of the pixel's square footprint in the plane normal
    to the view axis at the sample's depth: (sqrt(2)/2) * z * 2 tan(fovy/2) / H, z the depth along
    the view axis (computed here from the textbook projection)."""
    W, H = 64, 48
    rgba, depth = _img(H, W, 3)
    cam = synth.look_at((0.5, 0.5, 2.0), (0.5, 0.5, 0.5), (0, 1, 0), 30.0, W, H)
    sp = orc.unproject(rgba, depth, cam)
    F = np.array(cam.fwd, np.float64)
    eye = np.array(cam.eye, np.float64)
    z = (sp.pos_r[:, :3].astype(np.float64) - eye) @ F
    expected = math.sqrt(2) / 2 * z * 2 * cam.tan_half_fovy / H
    assert np.allclose(sp.pos_r[:, 3], expected, rtol=2e-6)


def test_voxel_radius_is_half_voxel_diagonal(orc):
    """The paper's own rule (§4.1): radius = half the length of a voxel's diagonal."""
    n = 256
    diag = np.float32(math.sqrt(3) / n)
    rgba, depth = _img(8, 8, 4)
    sp = orc.unproject(rgba, depth, synth.server_camera(1.4, 30.0, 8, 8), orc.RADIUS_VOXEL, diag)
    assert np.all(sp.pos_r[:, 3] == np.float32(diag * np.float32(0.5)))
    with open(os.path.join(GOLDEN, "paper_facts.json")) as f:
        facts = json.load(f)
    assert facts["radius_rule"]["fraction_of_voxel_diagonal"] == 0.5


def test_server_view_reproduced_by_warped_splats(orc):
    """Warping to the server's own camera must give back the server image: with footprint radii
    each pixel's ray hits its own sphere (through the centre) and misses the neighbours' (their
    centres lie more than a radius away from the ray for fields of view up to about 60 deg)."""
    for seed, (W, H, fovy) in enumerate([(64, 48, 30.0), (50, 50, 45.0)]):
        rgba, depth = _img(H, W, 10 + seed)
        cam = synth.look_at((0.5, 0.45, 1.9), (0.5, 0.5, 0.5), (0, 1, 0), fovy, W, H)
        sp = orc.unproject(rgba, depth, cam)
        out = orc.trace(orc.Scene(sp), cam)
        assert out["nhits"].max() == 1
        assert np.abs(out["rgba"] - rgba.reshape(-1, 4).astype(np.float64)).max() < 1e-12


def test_tiny_workload_view_reproduction(orc):
    W = synth.TINY
    cam = W.server_cam()
    rgba, depth = orc.raycast(W.volume(), synth.tf_ramp(), cam)
    srv = rgba.astype(np.float32)
    sp = orc.unproject(srv, depth, cam)
    assert sp.n > 5000
    out = orc.trace(orc.Scene(sp), cam)
    assert np.abs(out["rgba"] - srv.reshape(-1, 4)).max() < 1e-12


# ----------------------------------------------------------------------------------------------
# volume ray caster
# ----------------------------------------------------------------------------------------------
def _axis_cam(n_pix=5, dist=2.0):
    return synth.look_at((0.5, 0.5, 0.5 + dist), (0.5, 0.5, 0.5), (0, 1, 0), 10.0, n_pix, n_pix)


def _tf_const(alpha, rgb=(0.3, 0.6, 0.9)):
    tf = np.zeros((256, 4), np.float32)
    tf[:, :3] = rgb
    tf[:, 3] = alpha
    return tf


def test_homogeneous_volume_closed_form(orc):
    """Constant opacity alpha along the centre ray: m samples fit in the cube (t_in = D - 1/2,
    t_out = D + 1/2, spacing step/n), A = 1 - (1 - alpha)^(step * m) and C = rgb * A."""
    n, a = 16, 0.05
    vol = np.full((n, n, n), 0.5, np.float32)
    tf = _tf_const(a)
    cam = _axis_cam(5, 2.0)
    rgba, depth = orc.raycast(vol, tf, cam, step_vox=0.5, tau=0.01)
    dt = 0.5 / n
    m = int(math.floor(1.0 / dt - 0.5)) + 1  # j with (j + 1/2) dt < 1
    A = 1 - (1 - a) ** (0.5 * m)
    c = rgba[2, 2]
    assert abs(c[3] - A) < 1e-6
    assert np.allclose(c[:3], np.array([0.3, 0.6, 0.9], np.float32) * A, atol=1e-6)
    assert abs(depth[2, 2] - (2.0 - 0.5 + 0.5 * dt)) < 1e-6  # first sample already above tau


def test_empty_volume_gives_holes(orc):
    vol = np.zeros((8, 8, 8), np.float32)
    rgba, depth = orc.raycast(vol, synth.tf_ramp(), _axis_cam(6))
    assert np.all(rgba == 0) and np.all(np.isinf(depth))


def test_ray_missing_the_cube(orc):
    cam = synth.look_at((3.0, 3.0, 3.0), (4.0, 4.0, 4.0), (0, 1, 0), 10.0, 4, 4)
    rgba, depth = orc.raycast(np.ones((4, 4, 4), np.float32), synth.tf_ramp(), cam)
    assert np.all(rgba == 0) and np.all(np.isinf(depth))


@pytest.mark.parametrize("n", [16, 32])
def test_step_volume_threshold_crossing(orc, n):
    """Value 0 in the far half (z < 1/2), 1 in the near half along a ray looking down -z: the
    trilinear value between the two centre slices rises linearly, so alpha (= value for the ramp)
    first reaches tau at z = (n/2 + 1/2 - tau) / n ... measured from the near side it is the
    first sample past the point where the ramp between slice centres passes tau."""
    vol = np.zeros((n, n, n), np.float32)
    vol[n // 2:] = 1.0   # z >= 1/2 (near the camera at +z) is dense
    tau = 0.3
    cam = _axis_cam(3, 2.0)
    _, depth = orc.raycast(vol, synth.tf_ramp(), cam, step_vox=0.5, tau=tau)
    # along the centre ray z = 2.5 - t; the near half is fully dense: first sample has alpha = 1
    dt = 0.5 / n
    assert abs(depth[1, 1] - (2.0 - 0.5 + 0.5 * dt)) < 1e-6
    # flip: dense far half, the ray enters empty space and crosses the ramp
    vol2 = vol[::-1].copy()
    _, depth2 = orc.raycast(vol2, synth.tf_ramp(), cam, step_vox=0.5, tau=tau)
    # slice centres z_i = (i + 1/2)/n; value(z) = 1 for z <= z_{n/2-1}, 0 for z >= z_{n/2},
    # linear between: value = (z_{n/2} - z) * n.  value >= tau  <=>  z <= z_{n/2} - tau/n
    z_cross = (n // 2 + 0.5) / n - tau / n
    t_cross = 2.5 - z_cross
    t_in = 2.0 - 0.5
    j = math.ceil((t_cross - t_in) / dt - 0.5)
    assert abs(depth2[1, 1] - (t_in + (j + 0.5) * dt)) < 1e-6


def test_fallback_depth_first_nonzero_sample(orc):
    """No sample reaches tau but some have alpha > 0: the depth is the first such sample."""
    n = 16
    vol = np.zeros((n, n, n), np.float32)
    vol[: n // 2] = 0.05   # far half faintly dense, alpha = 0.05 < tau
    cam = _axis_cam(3, 2.0)
    rgba, depth = orc.raycast(vol, synth.tf_ramp(), cam, step_vox=0.5, tau=0.1)
    dt = 0.5 / n
    # value > 0 as soon as the trilinear ramp between slice n/2 and n/2-1 starts: z < z_{n/2}
    z0 = (n // 2 + 0.5) / n
    t_in = 1.5
    j = math.floor((2.5 - z0 - t_in) / dt - 0.5) + 1
    assert abs(depth[1, 1] - (t_in + (j + 0.5) * dt)) < 1e-6
    assert 0 < rgba[1, 1, 3] < 1


def test_u8_volume_matches_scaled_f32(orc):
    """A u8 volume is the same as the f32 volume of its counts / 255, up to binary32 rounding of the
    decision path; the binary64 composites agree to 1e-9."""
    rng = np.random.default_rng(5)
    v8 = rng.integers(0, 256, size=(12, 12, 12), dtype=np.uint8)
    v32 = (v8.astype(np.float64) / 255.0).astype(np.float32)
    cam = synth.look_at((1.5, 1.2, 2.0), (0.5, 0.5, 0.5), (0, 1, 0), 40.0, 12, 12)
    a, da = orc.raycast(v8, synth.tf_ramp(), cam)
    b, db = orc.raycast(v32, synth.tf_ramp(), cam)
    assert np.abs(a - b).max() < 1e-6


def test_raycast_pixel_subset_matches(orc):
    W = synth.TINY
    cam = W.server_cam()
    vol = W.volume()
    full_rgba, full_depth = orc.raycast(vol, synth.tf_ramp(), cam)
    pix = np.array([0, 777, 8000, 16383, 4242])
    r, d = orc.raycast(vol, synth.tf_ramp(), cam, pixels=pix)
    assert np.array_equal(r, full_rgba.reshape(-1, 4)[pix])
    assert np.array_equal(d, full_depth.reshape(-1)[pix])


def test_oracle_matches_frozen_golden(orc):
    """Regression pin: the oracle's tiny-workload values frozen by tests/golden/make_golden.py."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    with open(os.path.join(GOLDEN, "tiny_oracle.json")) as f:
        gold = json.load(f)
    now = mg.compute()
    assert now["n_splats"] == gold["n_splats"]
    for k in ("server_rgba", "server_depth", "client_rgba_all_hits", "client_rgba_first_hit"):
        assert np.allclose(np.array(now[k]), np.array(gold[k]), atol=1e-6), k
    assert abs(now["client_alpha_sum"] - gold["client_alpha_sum"]) < 1e-3
