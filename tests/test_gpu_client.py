"""The stream-pipelined client (host frame in, host views out) returns exactly the images of the
plain calls, across scene-slot reuse and ring wrap-around."""
import numpy as np
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


def test_pipeline_equals_plain_calls(wrs):
    from paper_2006_14726_b300.client import WarpingClient
    SW, SH, CW, CH = 160, 120, 144, 100
    base = synth.server_camera(1.4, 30.0, SW, SH)
    frames = []
    for g in range(5):
        rgba, depth = synth.synthetic_server_image(SW, SH, 900 + g)
        srv = base if g == 0 else synth.orbit(base, (0, 1, 0), 3.0 * g)
        frames.append((torch.from_numpy(rgba).pin_memory(), torch.from_numpy(depth).pin_memory(), srv))
    views = [synth.orbit(base, (0.6, 0.8, 0), 2.0 + v, CW, CH) for v in range(3)]
    params = wrs.TraceParams(width=4, k_chunk=2)
    client = WarpingClient(SW, SH, CW, CH, params, leaf_size=2, ring=4)
    got = []
    for hr, hd, srv in frames:
        client.submit(hr, hd, srv)
        tickets = [client.render(v) for v in views]
        got.append([client.result(t).clone() for t in tickets])
    # an uncollected wrap-around: more renders than the ring holds, collected at the end
    hr, hd, srv = frames[0]
    client.submit(hr, hd, srv)
    tickets = [client.render(views[i % 3]) for i in range(6)]
    late = [client.result(t).clone() for t in tickets[-4:]]
    with pytest.raises(ValueError):
        client.result(tickets[0])
    client.synchronize()
    wrs.check_status(client.status)
    for (hr, hd, srv), imgs in zip(frames, got):
        sp = wrs.unproject(hr.cuda(), hd.cuda(), srv)
        bvh, srt = wrs.build_lbvh(sp, 2)
        for v, img in zip(views, imgs):
            want = wrs.trace(bvh, srt, v, params).cpu()
            assert torch.equal(img, want)
    sp = wrs.unproject(frames[0][0].cuda(), frames[0][1].cuda(), frames[0][2])
    bvh, srt = wrs.build_lbvh(sp, 2)
    for i, img in zip(range(2, 6), late):
        assert torch.equal(img, wrs.trace(bvh, srt, views[i % 3], params).cpu())
