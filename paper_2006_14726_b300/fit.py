"""Fitting the per-splat radius scales to novel views, with checkpoint and resume.

The paper suggests taking the splat radius from the data rather than from a fixed rule (§6); the
differentiable renderer (wrs_trace_backward behind :mod:`.autograd`) makes that a gradient
descent: the radius scales s (r = max(s, 0) r0, compacted splat order) are moved by Adam to
lower the mean squared error between the rendered client views and reference images of the same
poses.  Every step refits the LBVH to the current scales (the splat centres do not move, so the
tree's order and shape stay; wrs_refit_lbvh), then one launch traces all views and one launch
runs the adjoint over all views.

With ``graph=True`` (CUDA only) the whole step — rebuild, trace, loss, adjoint and the Adam
update — is captured once in a CUDA graph and replayed: a step then costs one graph launch of
host time instead of the ~40 launches and the autograd bookkeeping that issuing it costs (the
step's GPU work is a couple of milliseconds, about what issuing it eagerly takes).  The first
GRAPH_WARMUP steps run eagerly (they warm the allocator and the autograd engine before the
capture); they are ordinary steps of the fit.

A fit can be checkpointed between steps (scales, Adam moments and step counts, the step index,
the loss history) and resumed in a new process; the resumed fit continues from the same state.
"""
from __future__ import annotations

import os
from typing import Callable, List, Optional, Sequence

import torch
import torch.nn.functional as F

from . import RefitTree, tree_layout
from .autograd import render_views

# eager steps before the capture of a graphed fit
GRAPH_WARMUP = 3


class RadiusFit:
    """Adam on the radius scales of one splat set against reference views.

    ``render``: optional callable scales -> images [V,H,W,4] (default: :func:`render_views` of
    ``splats`` with the fixed colours and opacities); the loss is mean((images - targets)^2).
    ``graph``: capture the step in a CUDA graph after GRAPH_WARMUP eager steps (CUDA only; the
    render callable must then launch its work on torch's current stream, read nothing back to
    the host and allocate the same buffers on every call)."""

    def __init__(self, splats, cams: Sequence, targets: torch.Tensor, params, leaf_size: int = 1,
                 lr: float = 1e-2, rgba: Optional[torch.Tensor] = None,
                 opacity: Optional[torch.Tensor] = None, scale: Optional[torch.Tensor] = None,
                 render: Optional[Callable[[torch.Tensor], torch.Tensor]] = None,
                 graph: bool = False):
        self.targets = targets
        self.lr = float(lr)
        if render is None:
            n = splats.count()
            dev = targets.device
            self.rgba = (rgba if rgba is not None else splats.rgba[:n].clone()).detach()
            self.opacity = (opacity if opacity is not None
                            else torch.ones(n, device=dev)).detach()
            cams = list(cams)
            self.tree = RefitTree(splats, leaf_size, layout=tree_layout(params))

            def render(s):
                return render_views(splats, cams, self.rgba, self.opacity, s, params, leaf_size,
                                    tree=self.tree)
        self.render = render
        if scale is None:
            n = splats.count() if splats is not None else targets.shape[0]
            scale = torch.ones(n, device=targets.device)
        self.scale = scale.detach().clone().requires_grad_(True)
        self.graph = bool(graph)
        if self.graph and not self.scale.is_cuda:
            raise ValueError("graph=True needs the scales on a CUDA device")
        self.opt = self._adam()
        self.step_index = 0
        self._losses: List[float] = []
        self._pending: List[torch.Tensor] = []  # device losses of steps not yet read back
        self._cuda_graph = None
        self._graph_loss = None
        self._warm = 0  # eager warm-up steps taken since the last (re)start of a graphed fit

    def _adam(self) -> torch.optim.Adam:
        if self.scale.is_cuda:
            # one fused kernel per update, its step count on the device (a graph may capture it)
            return torch.optim.Adam([self.scale], lr=self.lr, fused=True, capturable=True)
        return torch.optim.Adam([self.scale], lr=self.lr)

    @property
    def losses(self) -> List[float]:
        """Loss of every step so far, before that step's update (reads pending values back)."""
        if self._pending:
            self._losses.extend(torch.stack(self._pending).tolist())
            self._pending = []
        return self._losses

    def loss(self) -> torch.Tensor:
        return F.mse_loss(self.render(self.scale), self.targets)

    def _eager_step(self) -> torch.Tensor:
        self.opt.zero_grad(set_to_none=True)
        loss = self.loss()
        loss.backward()
        self.opt.step()
        return loss.detach()

    def _warm_step(self):
        # an eager step on a side stream: CUDA graph capture of autograd wants the engine and
        # the allocator warmed up off the capturing stream
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            loss = self._eager_step()
        torch.cuda.current_stream().wait_stream(side)
        self._warm += 1
        return loss

    def _capture(self):
        # the captured backward writes the gradient into the buffer it allocates during capture;
        # replays reuse it, so the gradient is never reset between replays
        self.opt.zero_grad(set_to_none=True)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            loss = self.loss()
            loss.backward()
            self.opt.step()
        self._cuda_graph, self._graph_loss = g, loss.detach()

    def _step_async(self):
        """One step without reading anything back: eager, or (graphed fit) one of the eager
        warm-up steps, else a replay of the captured step (captured first if need be)."""
        if not self.graph:
            loss = self._eager_step()
        elif self._cuda_graph is None and self._warm < GRAPH_WARMUP:
            loss = self._warm_step()
        else:
            if self._cuda_graph is None:
                self._capture()  # records the step without running it
            self._cuda_graph.replay()
            loss = self._graph_loss.clone()
        self._pending.append(loss)
        self.step_index += 1

    def step(self) -> float:
        """One Adam step; returns the loss before the step."""
        self._step_async()
        return self.losses[-1]

    def run(self, steps: int, checkpoint: Optional[str] = None, every: int = 0) -> List[float]:
        """``steps`` more steps; with ``checkpoint`` and ``every`` > 0, a checkpoint is written
        after every ``every``-th step (counted from the start of the fit).  The losses are read
        back once at the end (and at each checkpoint), not after every step."""
        start = self.step_index
        for _ in range(int(steps)):
            self._step_async()
            if checkpoint and every > 0 and self.step_index % every == 0:
                self.save(checkpoint)
        return self.losses[start:]

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
        self.opt = self._adam()
        self.opt.load_state_dict(sd["adam"])
        self.step_index = int(sd["step"])
        self._losses = list(sd["losses"])
        self._pending = []
        # a captured step refers to the previous optimizer's state: warm up and capture again
        self._cuda_graph = self._graph_loss = None
        self._warm = 0

    def save(self, path: str):
        """Write the checkpoint atomically (a crash leaves the previous one intact)."""
        tmp = f"{path}.tmp{os.getpid()}"
        torch.save(self.state_dict(), tmp)
        os.replace(tmp, path)

    def load(self, path: str):
        self.load_state_dict(torch.load(path, map_location="cpu", weights_only=True))
