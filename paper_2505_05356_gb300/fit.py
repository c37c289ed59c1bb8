"""The fitting iteration of the C-ToF Gaussian scene (Sec. 4), on the device.

One iteration: a fresh random background (Sec. 4, "Random background"),
deformation + projection of all frames, binning, compositing (Eq. 4), the
raw-sample L2 loss against the captured raw frames (the L_q term of Eq. 9,
without SSIM), the backward (Eq. S3 and the projection chain) and one fused
Adam update (betas (0.9, 0.999), epsilon 1e-15, Sec. 4 "Hyperparameters").
Every step is a library kernel that reads its iteration number from a
device-side state, so :meth:`FitLoop.capture` records the iteration once as a
CUDA graph and :meth:`FitLoop.run` replays it.

Learning rates: the paper gives the reflectivity rate (1.6e-4) and the MLP
rate (8e-4, used here for the trajectory coefficients that stand in for the
MLP offsets); the others follow the 3DGS defaults it builds on, converted to
the linear parameters this renderer takes (the scale rate 5e-3 on
log-scales times a typical scale of 0.05; the opacity rate 5e-2 on logits
times 0.2, about the sigmoid's slope of 0.25 at opacity 0.5).  The
projection box keeps opacity, scales and reflectivity valid.

Frame shards (several processes, one GPU each): a loop over frames
[frame_offset, frame_offset + B) of a batch of total_frames draws the
background values the whole batch's draw gives those frames, normalises the
loss by the whole batch's raw samples, and calls grad_hook on the parameter
gradients between the backward and the update -- `shard.allreduce_sum_`
sums them over the processes, so every process takes the same Adam step as
the unsharded loop.
"""
from __future__ import annotations

import math
from typing import Callable, Dict, Optional, Sequence

import torch

from . import gftorf

LEARNING_RATES: Dict[str, float] = {
    "means": 1.6e-4, "coeffs": 8e-4, "scales": 5e-3 * 0.05, "quats": 1e-3,
    "opacity": 5e-2 * 0.2, "amplitude": 1.6e-4,
}
BOUNDS = {"opacity": (1e-3, 1.0), "scales": (1e-5, 10.0), "amplitude": (0.0, 10.0)}


class FitLoop:
    """Device-resident fitting loop over a fixed batch of raw frames.

    params: the Gaussian parameters being fitted (float32 device tensors,
    updated in place); targets: (B, C, H, W) captured raw frames (only the
    raw channels enter the loss)."""

    def __init__(self, params: Dict[str, torch.Tensor], frames: Sequence[gftorf.Frame],
                 sensor: gftorf.Sensor, consts: gftorf.Consts, targets: torch.Tensor,
                 n_freq: int = 1, n_offsets: int = 4, tile=(16, 16), pixels_per_thread=4,
                 render_mode=1, seed: int = 0, lrs: Optional[Dict[str, float]] = None,
                 bounds=None, headroom: float = 1.5, flags: int = 0,
                 random_background: bool = True, frame_offset: int = 0,
                 total_frames: Optional[int] = None,
                 grad_hook: Optional[Callable[[Dict[str, torch.Tensor]], None]] = None):
        B, C, H, W = targets.shape
        total = B if total_frames is None else int(total_frames)
        if frame_offset < 0 or frame_offset + B > total:
            raise ValueError("frames [%d, %d) outside a batch of %d"
                             % (frame_offset, frame_offset + B, total))
        n = params["means"].shape[0]
        self.r = gftorf.Renderer(n, B, W, H, n_freq, n_offsets, tile=tile,
                                 render_mode=render_mode, pixels_per_thread=pixels_per_thread,
                                 flags=flags)
        if self.r.C != C:
            raise ValueError("targets have %d channels, the renderer %d" % (C, self.r.C))
        self.p, self.frames, self.sensor, self.consts = params, frames, sensor, consts
        self.targets = targets.contiguous()
        self.seed = seed
        self.random_background = random_background  # False: bg stays 0
        self.bg = torch.zeros((B, C), device=targets.device)
        self.r.fit_capacity(params, frames, sensor, consts, self.bg, headroom=headroom)
        self.out = torch.empty((B, C, H, W), device=targets.device)
        self.dout = torch.empty_like(self.out)
        self.lrs = dict(lrs or LEARNING_RATES)
        self.grads = self.r.alloc_grads(params, self.bg, want=list(self.lrs))
        self.opt = gftorf.Adam(params, self.lrs, bounds if bounds is not None else BOUNDS)
        self.state = gftorf.new_train_state(targets.device)
        self.graph = None
        self.update_graph = None
        # the shard's place in the whole batch (the defaults: the batch itself)
        self.bg_offset, self.bg_stride = frame_offset * C, total * C
        self.loss_count = (None if total == B else
                           float(total) * n_freq * n_offsets * H * W)
        self.grad_hook = grad_hook

    def param_grads(self) -> Dict[str, torch.Tensor]:
        """The gradients the update reads (what a grad_hook receives)."""
        return {k: self.grads[k] for k in self.opt.names}

    def forward_backward(self):
        """Enqueue an iteration up to the parameter gradients."""
        r = self.r
        gftorf.train_begin(self.state, self.bg if self.random_background else None, self.seed,
                           self.bg_offset, self.bg_stride)
        r.preprocess(self.p, self.frames, self.sensor, self.consts)
        r.bin()
        r.composite_fwd(self.bg, self.out)
        gftorf.l2_loss(r, self.out, self.targets, self.dout, self.state, count=self.loss_count)
        r.zero_grad_buffers(self.grads)
        r.composite_bwd(self.bg, self.dout, self.grads)
        r.preprocess_bwd(self.p, self.grads)

    def update(self):
        """Enqueue the Adam step from the current gradients."""
        self.opt.step(self.grads, self.state)

    def iteration(self):
        """Enqueue one iteration on the current stream (with grad_hook
        between the backward and the update)."""
        self.forward_backward()
        if self.grad_hook is not None:
            self.grad_hook(self.param_grads())
        self.update()

    def capture(self):
        """Record one iteration as a CUDA graph (runs nothing); with a
        grad_hook two graphs, the hook running between their replays."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        if self.grad_hook is None:
            with torch.cuda.graph(self.graph, stream=s):
                self.iteration()
            return self.graph
        with torch.cuda.graph(self.graph, stream=s):
            self.forward_backward()
        self.update_graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.update_graph, stream=s):
            self.update()
        return self.graph

    def run(self, k: int):
        """k iterations: graph replays when captured, else eager launches."""
        for _ in range(k):
            if self.graph is None:
                self.iteration()
            elif self.update_graph is None:
                self.graph.replay()
            else:
                self.graph.replay()
                self.grad_hook(self.param_grads())
                self.update_graph.replay()

    # --- checkpoint / resume ---------------------------------------------------
    def state_dict(self) -> Dict[str, object]:
        """Everything a resumed fit needs (host copies): the parameters, Adam's
        moments, the device iteration state (count and loss; the background
        of an iteration is a function of the seed and the count), the seed,
        learning rates and bounds.  torch.save-able."""
        torch.cuda.synchronize()
        host = lambda d: {k: v.detach().cpu().clone() for k, v in d.items() if v is not None}
        return {"params": host(self.p), "m": host(self.opt.m), "v": host(self.opt.v),
                "state": self.state.cpu().clone(), "seed": self.seed,
                "lrs": dict(self.lrs), "bounds": dict(self.opt.bounds)}

    def load_state_dict(self, sd: Dict[str, object]):
        """Restore into this loop's existing device buffers (a captured graph
        stays valid)."""
        for name, dst in (("params", self.p), ("m", self.opt.m), ("v", self.opt.v)):
            for k, t in sd[name].items():
                dst[k].copy_(t.to(dst[k].device))
        self.state.copy_(sd["state"].to(self.state.device))
        self.seed = int(sd["seed"])
        self.lrs.update(sd["lrs"])
        self.opt.lrs.update(sd["lrs"])
        self.opt.bounds.update(sd["bounds"])

    @property
    def step(self) -> int:
        return gftorf.train_step_count(self.state)

    def loss(self) -> float:
        """Loss of the last iteration (synchronises); a shard's part of the
        batch's loss (the parts add up to it)."""
        return gftorf.train_loss(self.state)

    def check(self):
        self.r.check()
        if not math.isfinite(self.loss()):
            raise FloatingPointError("non-finite loss")
