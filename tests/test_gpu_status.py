"""Device-side failure reporting: kernels turn impossible inputs and exceeded capacities into
status bits that the host reads, and the CUDA context stays usable.

Nothing here faults or hangs the GPU: a corrupted child reference is rejected by the traversal's
own range check before any access, a reference cycle is stopped by the per-pass visit budget, and
the backward pass stops a ray whose hit list needs more replay chunks than its table holds.
"""
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


def _scene(wrs, W=40, H=30, seed=2):
    rgba, depth = synth.synthetic_server_image(W, H, seed)
    srv = synth.server_camera(1.4, 30.0, W, H)
    sp = wrs.unproject(torch.from_numpy(rgba).cuda(), torch.from_numpy(depth).cuda(), srv)
    bvh, srt = wrs.build_lbvh(sp, 1)
    return bvh, srt, synth.orbit(srv, (0, 1, 0), 5.0)


def _child_refs(bvh, width):
    """The root's child references (int32 view): in its binary node (2), or its 4-wide node (4)."""
    if width == 2:
        return bvh.nodes[64 + 48:64 + 56].view(torch.int32)
    start = 64 + 64 * int(bvh.nodes[48:52].view(torch.int32).item())
    return bvh.nodes[start + 96:start + 112].view(torch.int32)


@pytest.mark.parametrize("schedule,width", [(0, 2), (1, 2), (0, 4), (1, 4), (2, 4)])
def test_corrupted_child_reference_sets_malformed_bit(wrs, schedule, width):
    bvh, srt, cam = _scene(wrs)
    params = wrs.TraceParams(schedule=schedule, width=width)
    good = wrs.trace(bvh, srt, cam, params).clone()
    bad = wrs.LBVH(bvh.capacity, 1)
    bad.nodes.copy_(bvh.nodes)
    _child_refs(bad, width)[0] = 0x7FFFFFF0  # an internal node far beyond the tree
    st = wrs.new_status()
    wrs.trace(bad, srt, cam, params, status=st)
    with pytest.raises(wrs.WrsError) as e:
        wrs.check_status(st)
    assert e.value.code == wrs.WRS_ERR_DEVICE and "malformed" in str(e.value)
    # a reference cycle (the root's child is the root) exhausts the visit budget
    bad.nodes.copy_(bvh.nodes)
    _child_refs(bad, width)[0] = 0
    wrs.trace(bad, srt, cam, params, status=st)
    with pytest.raises(wrs.WrsError):
        wrs.check_status(st)
    # the context is still usable and the good tree still gives the same image
    again = wrs.trace(bvh, srt, cam, params, status=st)
    wrs.check_status(st)
    assert torch.equal(again, good)


def test_backward_chunk_table_overflow_is_reported(wrs):
    """80 faint layers on every ray: with k_chunk = 1 the backward pass would need 80 replay
    chunks; its table holds 64, so it reports CHUNK_OVERFLOW and leaves those rays out."""
    W = H = 8
    layers = 80
    pos = np.zeros((layers * W * H, 4), np.float32)
    srv = synth.server_camera(1.4, 20.0, W, H)
    rgba = np.full((W * H, 4), 0.001, np.float32)
    depth = np.full((H, W), 1.2, np.float32)
    sp = wrs.unproject(torch.from_numpy(np.ascontiguousarray(rgba.reshape(H, W, 4))).cuda(),
                       torch.from_numpy(depth).cuda(), srv)
    # replicate the splats along each server ray at slightly increasing depths
    big = wrs.SplatBuffers(layers * W * H)
    p, c, i = (t.clone() for t in sp.view())
    n = p.shape[0]
    d = (p[:, :3] - torch.tensor(srv.eye, device="cuda")).contiguous()
    d = d / d.norm(dim=1, keepdim=True)
    for l in range(layers):
        big.pos_r[l * n:(l + 1) * n, :3] = p[:, :3] + d * (0.002 * l)
        big.pos_r[l * n:(l + 1) * n, 3] = p[:, 3] * 1.5
        big.rgba[l * n:(l + 1) * n] = c
        big.id[l * n:(l + 1) * n] = i + l * n
    big.n.fill_(layers * n)
    bvh, srt = wrs.build_lbvh(big, 1)
    st = wrs.new_status()
    img = wrs.trace(bvh, srt, srv, wrs.TraceParams(k_chunk=1), status=st)
    wrs.check_status(st)
    assert float(img[..., 3].max()) > 0.05  # many layers composited
    g = torch.ones(H, W, 4, device="cuda")
    for sched in (0, 1, 2):
        wrs.trace_backward(bvh, srt, srv, g, wrs.TraceParams(k_chunk=1, schedule=sched), status=st)
        with pytest.raises(wrs.WrsError) as e:
            wrs.check_status(st)
        assert "chunk" in str(e.value)
        # with k_chunk = 16 the same rays fit (80 hits = 5 chunks)
        wrs.trace_backward(bvh, srt, srv, g, wrs.TraceParams(k_chunk=16, schedule=sched), status=st)
        wrs.check_status(st)
