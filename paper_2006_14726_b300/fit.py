"""Fitting the per-splat radius scales to novel views, with checkpoint and resume.

The paper suggests taking the splat radius from the data rather than from a fixed rule (§6); the
differentiable renderer (wrs_trace_backward behind :mod:`.autograd`) makes that a gradient
descent: the radius scales s (r = max(s, 0) r0, compacted splat order) are moved by Adam to
lower the mean squared error between the rendered client views and reference images of the same
poses.  Every step is one LBVH rebuild with the current scales, one launch tracing all views and
one launch of the adjoint over all views.

A fit can be checkpointed between steps (scales, Adam moments and step counts, the step index,
the loss history) and resumed in a new process; the resumed fit continues from the same state.
"""
from __future__ import annotations

import os
from typing import Callable, List, Optional, Sequence

import torch

from .autograd import render_views


class RadiusFit:
    """Adam on the radius scales of one splat set against reference views.

    ``render``: optional callable scales -> images [V,H,W,4] (default: :func:`render_views` of
    ``splats`` with the fixed colours and opacities); the loss is mean((images - targets)^2)."""

    def __init__(self, splats, cams: Sequence, targets: torch.Tensor, params, leaf_size: int = 1,
                 lr: float = 1e-2, rgba: Optional[torch.Tensor] = None,
                 opacity: Optional[torch.Tensor] = None, scale: Optional[torch.Tensor] = None,
                 render: Optional[Callable[[torch.Tensor], torch.Tensor]] = None):
        self.targets = targets
        self.lr = float(lr)
        if render is None:
            n = splats.count()
            dev = targets.device
            self.rgba = (rgba if rgba is not None else splats.rgba[:n].clone()).detach()
            self.opacity = (opacity if opacity is not None
                            else torch.ones(n, device=dev)).detach()
            cams = list(cams)

            def render(s):
                return render_views(splats, cams, self.rgba, self.opacity, s, params, leaf_size)
        self.render = render
        if scale is None:
            n = splats.count() if splats is not None else targets.shape[0]
            scale = torch.ones(n, device=targets.device)
        self.scale = scale.detach().clone().requires_grad_(True)
        self.opt = torch.optim.Adam([self.scale], lr=self.lr)
        self.step_index = 0
        self.losses: List[float] = []

    def loss(self) -> torch.Tensor:
        return ((self.render(self.scale) - self.targets) ** 2).mean()

    def step(self) -> float:
        """One Adam step; returns the loss before the step."""
        self.opt.zero_grad(set_to_none=True)
        loss = self.loss()
        loss.backward()
        self.opt.step()
        self.step_index += 1
        val = float(loss.detach())
        self.losses.append(val)
        return val

    def run(self, steps: int, checkpoint: Optional[str] = None, every: int = 0) -> List[float]:
        """``steps`` more steps; with ``checkpoint`` and ``every`` > 0, a checkpoint is written
        after every ``every``-th step (counted from the start of the fit)."""
        out = []
        for _ in range(int(steps)):
            out.append(self.step())
            if checkpoint and every > 0 and self.step_index % every == 0:
                self.save(checkpoint)
        return out

    # -- checkpoint / resume -------------------------------------------------------------------
    def state_dict(self) -> dict:
        return {"version": 1, "step": self.step_index, "lr": self.lr,
                "scale": self.scale.detach().cpu().clone(),
                "adam": self.opt.state_dict(), "losses": list(self.losses)}

    def load_state_dict(self, sd: dict):
        if sd.get("version") != 1:
            raise ValueError("unknown checkpoint version")
        if sd["scale"].shape != self.scale.shape:
            raise ValueError(f"checkpoint holds {tuple(sd['scale'].shape)} scales, the fit "
                             f"{tuple(self.scale.shape)}")
        with torch.no_grad():
            self.scale.copy_(sd["scale"].to(self.scale.device))
        self.lr = float(sd["lr"])
        self.opt = torch.optim.Adam([self.scale], lr=self.lr)
        self.opt.load_state_dict(sd["adam"])
        self.step_index = int(sd["step"])
        self.losses = list(sd["losses"])

    def save(self, path: str):
        """Write the checkpoint atomically (a crash leaves the previous one intact)."""
        tmp = f"{path}.tmp{os.getpid()}"
        torch.save(self.state_dict(), tmp)
        os.replace(tmp, path)

    def load(self, path: str):
        self.load_state_dict(torch.load(path, map_location="cpu", weights_only=True))
