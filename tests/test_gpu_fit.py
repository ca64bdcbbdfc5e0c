"""The radius-scale fit on the GPU renderer: the loss falls, and a fit checkpointed mid-way and
resumed in a new fit object follows the uninterrupted one (up to the order of the float
atomics of the adjoint)."""
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


def _problem(wrs):
    rgba, depth = synth.synthetic_server_image(64, 64, 21, hole_frac=0.05)
    srv = synth.server_camera(1.4, 30.0, 64, 64)
    ref_sp = oracle.unproject(rgba, depth, srv)
    cams = [synth.orbit(srv, (0, 1, 0), 6.0), synth.orbit(srv, (1, 0, 0), -8.0)]
    # reference views: the oracle's render of the same splats with radius scale 1.4
    sc_true = np.full(ref_sp.n, 1.4, np.float32)
    ref = [oracle.trace(oracle.Scene(ref_sp, scale=sc_true, beta=0.25), c)["rgba"] for c in cams]
    targets = torch.tensor(np.stack(ref).reshape(2, 64, 64, 4), dtype=torch.float32, device="cuda")
    sp = wrs.unproject(torch.from_numpy(rgba).cuda(), torch.from_numpy(depth).cuda(), srv)
    params = wrs.TraceParams(edge_softness=0.25, k_chunk=4)
    return sp, cams, targets, params


def test_fit_resume_follows_uninterrupted(wrs, tmp_path):
    from paper_2006_14726_b300.fit import RadiusFit
    sp, cams, targets, params = _problem(wrs)
    a = RadiusFit(sp, cams, targets, params, 1, lr=1e-2)
    a.run(10)
    assert a.losses[-1] < 0.8 * a.losses[0]
    ck = str(tmp_path / "fit.pt")
    b = RadiusFit(sp, cams, targets, params, 1, lr=1e-2)
    b.run(4, checkpoint=ck, every=4)
    c = RadiusFit(sp, cams, targets, params, 1, lr=1e-2)
    c.load(ck)
    c.run(6)
    assert c.step_index == 10
    assert np.allclose(c.losses, a.losses, rtol=1e-4, atol=0)
    assert torch.allclose(c.scale, a.scale, rtol=1e-4, atol=1e-6)


def test_graphed_fit_follows_eager(wrs):
    """The step captured in a CUDA graph (rebuild, trace, loss, adjoint, Adam) and replayed
    takes the same steps as the eager fit: every replay renders with the scales the previous
    replay wrote."""
    from paper_2006_14726_b300.fit import GRAPH_WARMUP, RadiusFit
    sp, cams, targets, params = _problem(wrs)
    steps = GRAPH_WARMUP + 9
    a = RadiusFit(sp, cams, targets, params, 1, lr=1e-2)
    a.run(steps)
    g = RadiusFit(sp, cams, targets, params, 1, lr=1e-2, graph=True)
    g.run(steps)
    assert g._cuda_graph is not None and g.step_index == steps
    assert len(set(g.losses[GRAPH_WARMUP:])) == steps - GRAPH_WARMUP  # each replay a new step
    assert np.allclose(g.losses, a.losses, rtol=1e-4, atol=0)
    assert torch.allclose(g.scale, a.scale, rtol=1e-4, atol=1e-6)
    one = g.step()  # step() after run(): one more replay
    assert g.step_index == steps + 1 and one == g.losses[-1]


def test_graphed_fit_checkpoint_resume(wrs, tmp_path):
    """A graphed fit checkpointed after a few replays and resumed (warm-up and capture again in
    the new object) follows the uninterrupted graphed fit."""
    from paper_2006_14726_b300.fit import RadiusFit
    sp, cams, targets, params = _problem(wrs)
    a = RadiusFit(sp, cams, targets, params, 1, lr=1e-2, graph=True)
    a.run(14)
    ck = str(tmp_path / "fit.pt")
    b = RadiusFit(sp, cams, targets, params, 1, lr=1e-2, graph=True)
    b.run(6, checkpoint=ck, every=6)
    c = RadiusFit(sp, cams, targets, params, 1, lr=1e-2, graph=True)
    c.load(ck)
    c.run(8)
    assert c.step_index == 14
    assert np.allclose(c.losses, a.losses, rtol=1e-4, atol=0)
    assert torch.allclose(c.scale, a.scale, rtol=1e-4, atol=1e-6)
