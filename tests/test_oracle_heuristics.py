"""Oracle pins: the depth heuristics beyond first hit (§2, §5; readings: spec S2a).

A single ray along +x through the middle of a 32-voxel volume samples at the quarter-voxel offsets
c_i - 1/4 and c_i + 1/4 around each voxel centre c_i, so the sample that each heuristic must pick
follows by hand from the voxel values (trilinear reconstruction is linear between centres):
homogeneous media, a step, and a weak ramp followed by a jump.
"""
import numpy as np
import pytest

import synth

N = 32


def _ray_cam():
    # 1x1 image: the only ray is the view axis, o = (-1, 0.5, 0.5), d = (1, 0, 0); it enters the
    # unit cube at t = 1 and sample j sits at x = (j + 0.5) / 64
    return synth.look_at((-1.0, 0.5, 0.5), (2.0, 0.5, 0.5), (0, 0, 1), 30.0, 1, 1)


def _vol_x(values):
    v = np.asarray(values, np.float32)
    return np.ascontiguousarray(np.broadcast_to(v[None, None, :], (N, N, N)))


def _depth(orc, vol, heuristic, param=None, tau=0.1):
    rgba, depth = orc.raycast(vol, synth.tf_ramp(), _ray_cam(), 0.5, tau, heuristic=heuristic,
                              param=param)
    return float(depth.reshape(-1)[0]), rgba.reshape(-1, 4)[0]


def _t(j):
    return 1.0 + (j + 0.5) / 64.0


def test_sample_grid_is_as_assumed(orc):
    # first hit with tau = 0 on a constant medium: the first sample, x = 0.5 / 64
    d, _ = _depth(orc, _vol_x(np.full(N, 0.3)), orc.DEPTH_FIRST_HIT, 1e-6)
    assert abs(d - _t(0)) < 1e-6


def test_homogeneous_medium(orc):
    """alpha = 0.3 at every sample: contributions 0.3 * 0.7^j fall, so the first sample contributes
    most; accumulated opacity 1 - 0.7^(j+1) first reaches 0.5 at j = 1 (0.51); the gradient is 0
    everywhere, so its first maximum is the first sample."""
    vol = _vol_x(np.full(N, 0.3))
    assert abs(_depth(orc, vol, orc.DEPTH_MAX_CONTRIBUTION)[0] - _t(0)) < 1e-6
    assert abs(_depth(orc, vol, orc.DEPTH_ACCUMULATED, 0.5)[0] - _t(1)) < 1e-6
    assert abs(_depth(orc, vol, orc.DEPTH_ACCUMULATED, 0.8)[0] - _t(4)) < 1e-6  # 1 - 0.7^5 = 0.832
    assert abs(_depth(orc, vol, orc.DEPTH_MAX_GRADIENT)[0] - _t(0)) < 1e-6


def test_step_medium(orc):
    """0 before voxel 16, 0.6 from it: the samples around the step see alpha 0.15 (j = 31), 0.45
    (j = 32), then 0.6.  Contributions 0.15, 0.85 * 0.45 = 0.3825, 0.4675 * 0.6 = 0.2805: the
    maximum is j = 32; accumulated opacity 0.15 then 0.5325 >= 0.5 at j = 32; the gradient is 0.6
    at both j = 31 and j = 32 (first maximum: 31)."""
    vol = _vol_x([0.0] * 16 + [0.6] * 16)
    assert abs(_depth(orc, vol, orc.DEPTH_FIRST_HIT)[0] - _t(31)) < 1e-6
    assert abs(_depth(orc, vol, orc.DEPTH_MAX_CONTRIBUTION)[0] - _t(32)) < 1e-6
    assert abs(_depth(orc, vol, orc.DEPTH_ACCUMULATED, 0.5)[0] - _t(32)) < 1e-6
    assert abs(_depth(orc, vol, orc.DEPTH_MAX_GRADIENT)[0] - _t(31)) < 1e-6


def test_gradient_finds_the_jump_after_a_weak_ramp(orc):
    """0.2 + 0.01 i up to voxel 15, then 0.9: first hit (tau 0.1) takes the first sample, the
    gradient peaks at the jump: central differences one voxel apart give 0.56 - 0.01 f just after
    the centre c_15 (f = offset in voxels) and 0.56 - 0.54 f just before it, so j = 31 (c_15 + 1/4)
    beats j = 30 (c_15 - 1/4) and j = 32 (c_15 + 3/4)."""
    vol = _vol_x([0.2 + 0.01 * i for i in range(16)] + [0.9] * 16)
    assert abs(_depth(orc, vol, orc.DEPTH_FIRST_HIT)[0] - _t(0)) < 1e-6
    assert abs(_depth(orc, vol, orc.DEPTH_MAX_GRADIENT)[0] - _t(31)) < 1e-6


def test_fallbacks_and_colour_independence(orc):
    # accumulated opacity never reaches theta: the first sample with alpha > 0
    thin = _vol_x(np.full(N, 0.001))
    assert abs(_depth(orc, thin, orc.DEPTH_ACCUMULATED, 0.5)[0] - _t(0)) < 1e-6
    empty = _vol_x(np.zeros(N))
    for h in (orc.DEPTH_MAX_CONTRIBUTION, orc.DEPTH_ACCUMULATED, orc.DEPTH_MAX_GRADIENT):
        assert _depth(orc, empty, h)[0] == np.inf
    # the heuristic picks the depth only: the composite is the same for all of them
    vol = _vol_x([0.2 + 0.01 * i for i in range(16)] + [0.9] * 16)
    cols = [_depth(orc, vol, h)[1] for h in range(4)]
    for c in cols[1:]:
        assert np.array_equal(c, cols[0])


@pytest.mark.parametrize("h", [1, 2, 3])
def test_heuristic_images_on_a_blob_volume(orc, h):
    """On a real volume every heuristic keeps the first-hit rule's set of pixels with a depth (a
    depth exists iff some sample has alpha > 0) and puts the depth on a sample inside the cube."""
    W = synth.TINY
    cam = W.server_cam()
    vol = W.volume()
    _, d0 = orc.raycast(vol, synth.tf_ramp(), cam)
    _, dh = orc.raycast(vol, synth.tf_ramp(), cam, heuristic=h)
    assert np.array_equal(np.isfinite(d0), np.isfinite(dh))
    eye = np.array(cam.eye)
    dist_far = np.linalg.norm(eye - 0.5) + 0.9
    assert np.all(dh[np.isfinite(dh)] <= dist_far)
    # no heuristic picks a sample before the pixel's first sample with alpha > 0
    _, d_any = orc.raycast(vol, synth.tf_ramp(), cam, tau=1e-30)
    fin = np.isfinite(d_any)
    assert np.all(dh[fin] >= d_any[fin])
