"""Oracle pins: accumulation of several server frames into one splat set (future work, §6; reading:
spec S3a).

Expected values come from the server images themselves (which pixels carry a sample, their ids),
exact binary32 scalings by powers of two, the closed form of compositing a sphere twice, and the
first-hit rule on duplicated spheres -- never from the oracle's own accumulation code.
"""
import numpy as np

import synth


def _frame(W, H, seed, cam_seed=None):
    rgba, depth = synth.synthetic_server_image(W, H, seed)
    cam = synth.server_camera(1.4, 30.0, W, H)
    if cam_seed is not None:
        cam = synth.poses_in_cap(cam, 1, 10.0, cam_seed, W, H)[0]
    return rgba, depth, cam


def _keep(rgba, depth):
    return np.flatnonzero((np.isfinite(depth) & (depth >= 0) & (rgba[..., 3] > 0)).reshape(-1))


def test_window_layout_ids_and_weights(orc):
    """Newest frame first with ids = pixel index; the frame of age g after it with ids shifted by
    g * Ws * Hs and colours scaled by decay^g (0.5^g is exact in binary32)."""
    W, H = 31, 23
    frames = [_frame(W, H, 10 + g, cam_seed=20 + g) for g in range(3)]
    acc = orc.accumulate(frames, decay=0.5)
    npix = W * H
    ids, cols = [], []
    for g, (rgba, depth, _) in enumerate(frames):
        k = _keep(rgba, depth)
        ids.append(k + g * npix)
        cols.append(rgba.reshape(-1, 4)[k] * np.float32(0.5 ** g))
    assert acc.n == sum(len(i) for i in ids)
    assert np.array_equal(acc.id, np.concatenate(ids).astype(np.uint32))
    assert np.array_equal(acc.rgba.view(np.uint32), np.concatenate(cols).astype(np.float32).view(np.uint32))
    # every record lies on its own frame's server ray at that pixel's depth (Eq. 1)
    off = 0
    for g, (rgba, depth, cam) in enumerate(frames):
        k = _keep(rgba, depth)
        eye = np.array(cam.eye, np.float64)
        p = acc.pos_r[off:off + len(k), :3].astype(np.float64)
        t = depth.reshape(-1)[k].astype(np.float64)
        assert np.all(np.abs(np.linalg.norm(p - eye, axis=1) - t) < 2e-6 * (1 + t))
        off += len(k)


def test_window_weights_are_powers():
    import oracle
    assert np.array_equal(oracle.window_weights(4, 0.5), np.float32([1, 0.5, 0.25, 0.125]))
    assert np.array_equal(oracle.window_weights(3), np.ones(3, np.float32))
    w = oracle.window_weights(6, 0.9).astype(np.float64)
    assert np.allclose(w, 0.9 ** np.arange(6), rtol=1e-6, atol=0)


def test_capacity_drops_the_tail_and_flags(orc):
    W, H = 20, 12
    a, b = _frame(W, H, 3), _frame(W, H, 4, cam_seed=5)
    full, ovf = orc.append_frame(None, *a)
    full, ovf2 = orc.append_frame(full, *b, id_base=W * H)
    assert not ovf and not ovf2
    n = full.n
    cut, o = orc.append_frame(None, *a, capacity=n - 7)
    cut, o2 = orc.append_frame(cut, *b, id_base=W * H, capacity=n - 7)
    assert o2 and cut.n == n - 7
    assert np.array_equal(cut.id, full.id[:n - 7])
    assert np.array_equal(cut.pos_r.view(np.uint32), full.pos_r[:n - 7].view(np.uint32))
    exact, o3 = orc.append_frame(orc.append_frame(None, *a, capacity=n)[0], *b, id_base=W * H,
                                 capacity=n)
    assert not o3 and exact.n == n


def test_newest_frame_wins_equal_depth_first_hit(orc):
    """Two frames with the same depth image and camera give coincident spheres; with H = 1 the
    (key, id) order picks the newer frame's copy (smaller ids), so the image is the newer frame's
    alone -- a frame order or id offset the wrong way round shows the older colours."""
    W, H = 24, 18
    rgba, depth, cam = _frame(W, H, 7)
    newer = (rgba * np.float32(0.5)).astype(np.float32)
    acc = orc.accumulate([(newer, depth, cam), (rgba, depth, cam)])
    ccam = synth.orbit(cam, (0, 1, 0), 4.0, 32, 24)
    one = orc.trace(orc.Scene(orc.unproject(newer, depth, cam), max_hits=1), ccam)
    two = orc.trace(orc.Scene(acc, max_hits=1), ccam)
    assert np.array_equal(two["rgba"], one["rgba"])
    assert np.array_equal(two["hash"], one["hash"])
    assert np.array_equal(two["nhits"], 2 * one["nhits"])


def test_doubled_frame_composites_each_sphere_twice(orc):
    """H = 0: a ray that meets one sphere of a frame meets its copy too; front to back,
    C = c + (1 - a) c = (2 - a) c and 1 - T = 1 - (1 - a)^2 (hard edges, unit opacity)."""
    W, H = 24, 18
    rgba, depth, cam = _frame(W, H, 8)
    acc = orc.accumulate([(rgba, depth, cam), (rgba, depth, cam)])
    ccam = synth.orbit(cam, (0, 1, 0), 3.0, 40, 30)
    one = orc.trace(orc.Scene(orc.unproject(rgba, depth, cam)), ccam)
    two = orc.trace(orc.Scene(acc), ccam)
    assert np.array_equal(two["nhits"], 2 * one["nhits"])
    single = (one["nhits"] == 1) & (one["nused"] == 1)
    assert single.sum() > 20
    a = one["rgba"][single, 3]
    assert np.allclose(two["rgba"][single, :3], (2 - a)[:, None] * one["rgba"][single, :3],
                       rtol=1e-12, atol=1e-15)
    assert np.allclose(two["rgba"][single, 3], 1 - (1 - a) ** 2, rtol=1e-12, atol=1e-15)
