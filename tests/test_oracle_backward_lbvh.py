"""Oracle pins: the adjoint of the ordered compositing (spec S7) against central finite
differences of the oracle's own forward, and the LBVH reference (§4.1, §4.2) against the
defining properties of Morton codes and of the binary radix tree.
"""
import numpy as np
import pytest

import synth


def _scene(orc, W=24, H=24, seed=0, beta=0.25):
    rgba, depth = synth.synthetic_server_image(W, H, seed, hole_frac=0.1)
    srv = synth.look_at((0.5, 0.5, 1.9), (0.5, 0.5, 0.5), (0, 1, 0), 30.0, W, H)
    sp = orc.unproject(rgba, depth, srv)
    rng = np.random.default_rng(seed)
    scale = rng.uniform(1.0, 2.5, sp.n).astype(np.float32)     # overlapping spheres
    opacity = rng.uniform(0.3, 1.0, sp.n).astype(np.float32)
    cli = synth.orbit(srv, (0.3, 1.0, 0.0), 12.0)
    return sp, scale, opacity, cli


def _loss_and_fwd(orc, sp, scale, opacity, cam, w, beta):
    sc = orc.Scene(sp, scale=scale, opacity=opacity, beta=beta)
    out = orc.trace(sc, cam, bvh=None)
    return float(np.sum(out["rgba"] * w)), out


@pytest.mark.parametrize("beta", [0.25, 0.0])
def test_adjoint_matches_central_differences(orc, beta):
    sp, scale, opacity, cam = _scene(orc, beta=beta)
    rng = np.random.default_rng(1)
    w = rng.normal(size=(cam.width * cam.height, 4))
    L0, base = _loss_and_fwd(orc, sp, scale, opacity, cam, w, beta)
    sc = orc.Scene(sp, scale=scale, opacity=opacity, beta=beta)
    g_rgba, g_op, g_sc = orc.trace_backward(sc, cam, w, bvh=None)
    if beta == 0.0:
        assert np.all(g_sc == 0)
    h = 1e-3
    checked = {"rgba": 0, "op": 0, "sc": 0}
    skipped = 0

    def fd(mutate):
        nonlocal skipped
        vals = []
        for sgn in (+1, -1):
            s2, sc2, op2 = mutate(sgn)
            L, o = _loss_and_fwd(orc, s2, sc2, op2, cam, w, beta)
            if not (np.array_equal(o["hash"], base["hash"]) and np.array_equal(o["nused"], base["nused"])):
                skipped += 1
                return None  # the perturbation changed a hit list: not differentiable there
            vals.append(L)
        return (vals[0] - vals[1]) / (2 * h)

    idx = rng.choice(sp.n, size=min(40, sp.n), replace=False)
    for i in idx:
        for ch in range(4):
            def m(sgn, i=i, ch=ch):
                rgba = sp.rgba.copy()
                rgba[i, ch] = np.float32(rgba[i, ch] + sgn * h)
                return orc.Splats(sp.pos_r, rgba, sp.id), scale, opacity
            # the perturbation is rounded to binary32: divide by the realised step
            step = float(np.float32(sp.rgba[i, ch] + h)) - float(np.float32(sp.rgba[i, ch] - h))
            g = fd(m)
            if g is None:
                continue
            g *= 2 * h / step
            assert abs(g - g_rgba[i, ch]) <= 1e-2 * max(1e-3, abs(g)), (i, ch, g, g_rgba[i, ch])
            checked["rgba"] += 1

        def mo(sgn, i=i):
            op = opacity.copy()
            op[i] = np.float32(op[i] + sgn * h)
            return sp, scale, op
        x = float(opacity[i]) * float(sp.rgba[i, 3])
        step = float(np.float32(opacity[i] + h)) - float(np.float32(opacity[i] - h))
        g = fd(mo)
        if g is not None and abs(x - 1) > 2e-3:
            g *= 2 * h / step
            assert abs(g - g_op[i]) <= 1e-2 * max(1e-3, abs(g)), (i, g, g_op[i])
            checked["op"] += 1

        def ms(sgn, i=i):
            s = scale.copy()
            s[i] = np.float32(s[i] + sgn * h)
            return sp, s, opacity
        step = float(np.float32(scale[i] + h)) - float(np.float32(scale[i] - h))
        g = fd(ms)
        if g is not None:
            g *= 2 * h / step
            assert abs(g - g_sc[i]) <= 1e-2 * max(1e-3, abs(g)), (i, g, g_sc[i])
            checked["sc"] += 1
    assert checked["rgba"] >= 100 and checked["op"] >= 20 and checked["sc"] >= 15, (checked, skipped)
    if beta > 0:
        assert np.abs(g_sc).max() > 0


def test_backward_zero_upstream_gives_zero(orc):
    sp, scale, opacity, cam = _scene(orc)
    sc = orc.Scene(sp, scale=scale, opacity=opacity, beta=0.25)
    g = orc.trace_backward(sc, cam, np.zeros((cam.width * cam.height, 4)), bvh=None)
    assert all(np.all(x == 0) for x in g)


def test_backward_bvh_equals_brute(orc):
    sp, scale, opacity, cam = _scene(orc, seed=3)
    sc = orc.Scene(sp, scale=scale, opacity=opacity, beta=0.25)
    w = np.random.default_rng(2).normal(size=(cam.width * cam.height, 4))
    a = orc.trace_backward(sc, cam, w, bvh=None)
    b = orc.trace_backward(sc, cam, w)
    for x, y in zip(a, b):
        assert np.allclose(x, y, rtol=1e-12, atol=1e-14)


# ----------------------------------------------------------------------------------------------
# LBVH reference
# ----------------------------------------------------------------------------------------------
def _compact(code):
    """Inverse of the 3-way bit interleave: (qx, qy, qz) with x on the highest bit of each triple."""
    q = [0, 0, 0]
    for b in range(10):
        for a in range(3):
            q[a] |= ((int(code) >> (3 * b + 2 - a)) & 1) << b
    return q


def _random_points(n, seed, dup_frac=0.0):
    rng = np.random.default_rng(seed)
    pos_r = np.zeros((n, 4), np.float32)
    pos_r[:, :3] = rng.uniform(0.1, 0.9, (n, 3))
    pos_r[:, 3] = rng.uniform(0.001, 0.01, n)
    if dup_frac > 0:  # duplicated centres exercise the index tie-break
        k = int(n * dup_frac)
        pos_r[rng.choice(n, k), :3] = pos_r[0, :3]
    return pos_r


@pytest.mark.parametrize("n,seed,dup", [(1000, 0, 0.0), (777, 1, 0.2), (64, 2, 0.5)])
def test_morton_codes_decode_to_the_cell_of_the_point(orc, n, seed, dup):
    pos_r = _random_points(n, seed, dup)
    ref = orc.lbvh(pos_r)
    order = ref["order"].astype(np.int64)
    assert np.array_equal(np.sort(order), np.arange(n))
    codes = ref["codes"].astype(np.int64)
    assert np.all(np.diff(codes) >= 0)
    same = np.diff(codes) == 0
    assert np.all(np.diff(order)[same] > 0)  # stable: equal codes keep index order
    lo = ref["cbounds"][:3].astype(np.float64)
    ext = ref["cbounds"][3:].astype(np.float64) - lo
    for k in range(n):
        q = _compact(codes[k])
        c = pos_r[order[k], :3].astype(np.float64)
        for a in range(3):
            cell_lo = lo[a] + q[a] * ext[a] / 1024
            cell_hi = lo[a] + (q[a] + 1) * ext[a] / 1024
            assert cell_lo - 1e-6 <= c[a] <= cell_hi + 1e-6


def _check_radix_tree(ref, M):
    codes = ref["codes"]
    child = ref["child"]
    if M == 1:
        assert ref["root"] == -(2 ** 31)
        return
    assert ref["root"] == 0
    # ranges bottom-up
    rng = {}

    def span(ref_):
        if ref_ < 0:
            j = ref_ & 0x7FFFFFFF
            return j, j
        a0, b0 = span(int(child[ref_, 0]))
        a1, b1 = span(int(child[ref_, 1]))
        assert b0 + 1 == a1  # children cover adjacent ranges
        rng[ref_] = (a0, b1)
        return a0, b1

    import sys
    sys.setrecursionlimit(10000)
    a, b = span(0)
    assert (a, b) == (0, M - 1)
    assert len(rng) == M - 1  # every internal node reached exactly once
    seen = []
    for i in range(M - 1):
        for c in child[i]:
            if c < 0:
                seen.append(int(c) & 0x7FFFFFFF)
    assert sorted(seen) == list(range(M))
    return rng, codes


@pytest.mark.parametrize("n,leaf,dup", [(500, 1, 0.0), (500, 1, 0.3), (999, 4, 0.0), (130, 8, 0.4), (3, 4, 0.0)])
def test_radix_tree_properties(orc, n, leaf, dup):
    pos_r = _random_points(n, 7, dup)
    ref = orc.lbvh(pos_r, leaf=leaf)
    M = (n + leaf - 1) // leaf
    res = _check_radix_tree(ref, M)
    if res is None:
        return
    rng, codes = res
    lkey = [(int(codes[j * leaf]) << 32) | j for j in range(M)]  # index-augmented leaf keys
    for i, (a, b) in rng.items():
        assert i == a or i == b  # the node index is one end of its range (Karras numbering)
        l_ref = int(ref["child"][i, 0])
        la, lb = (l_ref & 0x7FFFFFFF, l_ref & 0x7FFFFFFF) if l_ref < 0 else rng[l_ref]
        g = lb
        # the split is where the highest bit differing across the range flips
        top = (lkey[a] ^ lkey[b]).bit_length() - 1
        assert (lkey[g] >> top) & 1 == 0 and (lkey[g + 1] >> top) & 1 == 1


def test_lbvh_boxes_contain_spheres_tightly(orc):
    n, leaf = 400, 2
    pos_r = _random_points(n, 9)
    scale = np.random.default_rng(9).uniform(0.5, 2.0, n).astype(np.float32)
    ref = orc.lbvh(pos_r, scale=scale, leaf=leaf)
    order = ref["order"]
    child, boxes = ref["child"], ref["boxes"]
    r = (scale * pos_r[:, 3]).astype(np.float32).astype(np.float64)
    c = pos_r[:, :3].astype(np.float64)

    def leaves_of(ref_):
        if ref_ < 0:
            j = ref_ & 0x7FFFFFFF
            return list(order[j * leaf:(j + 1) * leaf])
        return leaves_of(int(child[ref_, 0])) + leaves_of(int(child[ref_, 1]))

    for i in range(len(child)):
        for s in range(2):
            prims = leaves_of(int(child[i, s]))
            lo = boxes[i, s, :3].astype(np.float64)
            hi = boxes[i, s, 3:].astype(np.float64)
            tight_lo = np.min(c[prims] - r[prims, None], axis=0)
            tight_hi = np.max(c[prims] + r[prims, None], axis=0)
            assert np.all(lo <= tight_lo) and np.all(hi >= tight_hi)
            assert np.all(lo >= np.nextafter(tight_lo.astype(np.float32), -np.inf) - 1e-12)
            assert np.all(hi <= np.nextafter(tight_hi.astype(np.float32), np.inf) + 1e-12)
