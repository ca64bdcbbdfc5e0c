"""The trace autotuner: it times every candidate launch, charges each the LBVH build of the layout
that launch needs (the 4-wide-only layout for the 4-wide traversal and the packet schedule, the
full layout for the binary traversal), returns the best by time + build share, and caches the
choice per workload signature.  The knobs never change results, so the tuned launch's image
equals any other launch's bitwise."""
import json

import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wrs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_14726_b300 as w
    return w


def test_tune_trace_charges_the_layouts_build(wrs, tmp_path, monkeypatch):
    from paper_2006_14726_b300 import autotune
    monkeypatch.setenv("WRS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    rgba, depth = synth.synthetic_server_image(160, 120, 17)
    srv = synth.server_camera(1.4, 30.0, 160, 120)
    sp = wrs.unproject(torch.from_numpy(rgba).cuda(), torch.from_numpy(depth).cuda(), srv)
    cams = [wrs.make_camera(synth.orbit(srv, (0, 1, 0), a, 96, 72)) for a in (3.0, -4.0)]
    best = autotune.tune_trace(sp, cams, leaves=(1, 2), ks=(1, 2), blocks=(128,), reps=1,
                               use_cache=True, build_weight=0.25)
    table = best["table"]
    # leaf x k x (one per-pixel block + persistent, each at widths 2 and 4, + packet at width 4)
    assert len(table) == 2 * 2 * (2 * 2 + 1)
    for leaf in (1, 2):
        rows = [r for r in table if r[0] == leaf]
        wide = {r[6] for r in rows if r[4] == 4 or r[3] == wrs.SCHEDULE_PACKET}
        full = {r[6] for r in rows if r[4] == 2 and r[3] != wrs.SCHEDULE_PACKET}
        assert len(wide) == 1 and len(full) == 1  # one build time per layout and leaf size
    scores = [r[5] + 0.25 * r[6] for r in table]
    assert best["score"] == pytest.approx(min(scores))
    # cached under the workload signature: the second call returns the stored choice
    stored = json.loads((tmp_path / "tune.json").read_text())
    assert len(stored) == 1
    again = autotune.tune_trace(sp, cams, leaves=(4,), ks=(8,), blocks=(64,), reps=1,
                                use_cache=True, build_weight=0.25)
    assert (again["leaf"], again["k_chunk"], again["width"]) == (best["leaf"], best["k_chunk"],
                                                               best["width"])
    # the tuned launch renders what any other launch renders
    p = wrs.TraceParams(0, 1e-5, 0.0, best["k_chunk"], best["block"], best["schedule"],
                        best["width"])
    bvh, srt = wrs.build_lbvh(sp, best["leaf"], layout=wrs.tree_layout(p))
    ref_bvh, ref_srt = wrs.build_lbvh(sp, 1)
    for c in cams:
        a = wrs.trace(bvh, srt, c, p)
        b = wrs.trace(ref_bvh, ref_srt, c, wrs.TraceParams(k_chunk=8, width=2))
        assert torch.equal(a.view(torch.int32), b.view(torch.int32))
