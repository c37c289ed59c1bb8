"""Steps streamed from host memory with the copies hidden behind compute.

Each step copies its inputs host -> device, runs the captured fwd+bwd, and
copies its outputs device -> host.  With two device buffer sets (one CUDA
graph per set) the host -> device copy of step i + 1 and the device -> host
copy of step i - 1 run on their own streams while step i computes; events
order every buffer reuse:

    h2d(i)      waits compute(i - 2)   (its set's inputs are free again)
    compute(i)  waits h2d(i), d2h(i - 2) (its set's outputs were read out)
    d2h(i)      waits compute(i)
"""
from __future__ import annotations

from typing import Callable, Dict, List

import torch


class HostStream:
    """`make_set()` returns one device buffer set: {"in": {name: tensor},
    "out": {name: tensor}, ...}; `step(bufs)` enqueues one step on the
    current stream reading bufs["in"] and writing bufs["out"] (it is captured
    once per set, so it must not allocate or synchronise)."""

    def __init__(self, make_set: Callable[[], Dict], step: Callable[[Dict], None], warmup: int = 2):
        self.sets: List[Dict] = [make_set(), make_set()]
        self.step = step
        self.h2d = torch.cuda.Stream()
        self.d2h = torch.cuda.Stream()
        self.loaded = [torch.cuda.Event() for _ in range(2)]
        self.computed = [torch.cuda.Event() for _ in range(2)]
        self.read = [torch.cuda.Event() for _ in range(2)]
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for bufs in self.sets:
                for _ in range(warmup):
                    step(bufs)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graphs = []
        for bufs in self.sets:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                step(bufs)
            self.graphs.append(g)
        torch.cuda.synchronize()

    def run(self, host_in: Dict[str, torch.Tensor], host_out: Dict[str, torch.Tensor],
            steps: int, start: torch.cuda.Event = None):
        """`steps` steps from the pinned host inputs into the pinned host
        outputs (the same host buffers every step).  The copy streams first
        wait for `start` (recorded on the current stream) if given; on return
        the current stream is ordered after the last copy out."""
        compute = torch.cuda.current_stream()
        if start is not None:
            self.h2d.wait_event(start)
            self.d2h.wait_event(start)
        for i in range(steps):
            k = i & 1
            bufs = self.sets[k]
            with torch.cuda.stream(self.h2d):
                self.h2d.wait_event(self.computed[k])
                for name, t in host_in.items():
                    bufs["in"][name].copy_(t, non_blocking=True)
                self.loaded[k].record(self.h2d)
            compute.wait_event(self.loaded[k])
            compute.wait_event(self.read[k])
            self.graphs[k].replay()
            self.computed[k].record(compute)
            with torch.cuda.stream(self.d2h):
                self.d2h.wait_event(self.computed[k])
                for name, t in host_out.items():
                    t.copy_(bufs["out"][name], non_blocking=True)
                self.read[k].record(self.d2h)
        compute.wait_stream(self.d2h)
        compute.wait_stream(self.h2d)
