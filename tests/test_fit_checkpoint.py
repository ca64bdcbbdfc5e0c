"""Checkpoint and resume of the radius-scale fit (RadiusFit), on the CPU: the render function is
a smooth stand-in for the renderer (the fit's bookkeeping does not depend on it), so an
interrupted and resumed fit must equal an uninterrupted one bitwise."""
import os

import pytest

torch = pytest.importorskip("torch")

from paper_2006_14726_b300.fit import RadiusFit  # noqa: E402


def _problem(seed=0, n=64):
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(2, 9, 7, 4, n, generator=g) / n ** 0.5
    target = torch.tanh(A @ (1.3 * torch.ones(n))) * 0.5

    def render(s):
        return torch.tanh(A @ s) * 0.5 + 0.01 * torch.sin(3 * s).mean()
    return render, target


def _fit(render, target, n=64):
    return RadiusFit(None, [], target, None, render=render, lr=1e-2, scale=torch.ones(n))


def test_resume_equals_uninterrupted(tmp_path):
    render, target = _problem()
    a = _fit(render, target)
    a.run(12)
    ck = str(tmp_path / "fit.pt")
    b = _fit(render, target)
    b.run(5, checkpoint=ck, every=5)
    assert os.path.exists(ck) and not any(p.name.startswith("fit.pt.tmp") for p in tmp_path.iterdir())
    c = _fit(render, target)  # a new fit object, as in a new process
    c.load(ck)
    assert c.step_index == 5 and c.losses == b.losses
    c.run(7)
    assert torch.equal(a.scale.detach(), c.scale.detach())
    assert a.losses == c.losses
    assert a.losses[-1] < a.losses[0]
    sa, sc = a.opt.state_dict()["state"][0], c.opt.state_dict()["state"][0]
    for k in ("exp_avg", "exp_avg_sq"):
        assert torch.equal(sa[k], sc[k])
    assert int(sa["step"]) == int(sc["step"]) == 12


def test_periodic_checkpoints_and_shape_check(tmp_path):
    render, target = _problem(1)
    ck = str(tmp_path / "fit.pt")
    f = _fit(render, target)
    f.run(9, checkpoint=ck, every=4)
    sd = torch.load(ck, weights_only=True)
    assert sd["step"] == 8 and len(sd["losses"]) == 8
    g = RadiusFit(None, [], target, None, render=render, scale=torch.ones(65))
    with pytest.raises(ValueError):
        g.load(ck)
    sd["version"] = 2
    with pytest.raises(ValueError):
        f.load_state_dict(sd)
