"""Launch-configuration autotuner for the batched fwd+bwd render.

Times one full step (preprocess, bin, composite, backward) of the caller's
actual problem for every valid (tile shape, pixels per thread, grid or
persistent compositing) and returns the fastest.  Results never change the
rendered values (the forward is bit-identical across these choices, the
gradients equal up to atomic summation order); only speed differs.
"""
from __future__ import annotations

import itertools
import json
import os
from typing import Dict, List, Optional, Sequence, Tuple

import torch

from . import gftorf

TILES: Tuple[Tuple[int, int], ...] = ((8, 8), (16, 16), (16, 32), (32, 32), (64, 32), (64, 64))
PIXELS_PER_THREAD = (1, 2, 4)
MODES = (0, 1)


def candidates(tiles=TILES, ppts=PIXELS_PER_THREAD, modes=MODES) -> List[dict]:
    out = []
    for (tw, th), ppt, mode in itertools.product(tiles, ppts, modes):
        if tw * th // ppt < 32:
            continue
        if tw >= 32 and ppt != 4:  # 32 wide or more: 4 pixels per thread only
            continue
        out.append(dict(tile=(tw, th), ppt=ppt, mode=mode))
    return out


def _step(r: gftorf.Renderer, params, frames, sensor, consts, bg, dout, out, grads):
    r.preprocess(params, frames, sensor, consts)
    r.bin()
    r.composite_fwd(bg, out)
    r.zero_grad_buffers(grads)
    r.composite_bwd(bg, dout, grads)
    r.preprocess_bwd(params, grads)


def time_config(cfg, n, n_frames, width, height, n_freq, n_offsets, params, frames,
                sensor, consts, bg, dout, steps=3, warmup=2, flags=0, n_sh=0) -> float:
    """Milliseconds per fwd+bwd step of one configuration (CUDA events)."""
    r = gftorf.Renderer(n, n_frames, width, height, n_freq, n_offsets, tile=cfg["tile"],
                        render_mode=cfg["mode"], pixels_per_thread=cfg["ppt"], flags=flags,
                        n_sh=n_sh)
    r.fit_capacity(params, frames, sensor, consts, bg)
    out = torch.empty((n_frames, r.C, height, width), dtype=r.torch_dtype, device=r.device)
    grads = r.alloc_grads(params, bg)
    for _ in range(warmup):
        _step(r, params, frames, sensor, consts, bg, dout, out, grads)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        _step(r, params, frames, sensor, consts, bg, dout, out, grads)
    e1.record()
    torch.cuda.synchronize()
    r.check()
    ms = e0.elapsed_time(e1) / steps
    del r, out, grads
    torch.cuda.empty_cache()
    return ms


def autotune(n, n_frames, width, height, n_freq, n_offsets, params, frames, sensor,
             consts, bg, dout, configs: Optional[Sequence[dict]] = None, steps=3,
             cache_path: Optional[str] = None, flags=0, n_sh=0) -> dict:
    """Fastest configuration for this problem: {'tile', 'ppt', 'mode', 'ms',
    'table'}.  With cache_path, results are read from / written to a JSON
    file keyed by the problem shape and device name."""
    key = "%s|n=%d|B=%d|%dx%d|F=%d|P=%d|flags=%d|sh=%d" % (
        torch.cuda.get_device_name(), n, n_frames, width, height, n_freq, n_offsets, flags, n_sh)
    cache: Dict[str, dict] = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            hit = dict(cache[key])
            hit["tile"] = tuple(hit["tile"])
            hit["cached"] = True
            return hit
    table = []
    for cfg in configs or candidates():
        ms = time_config(cfg, n, n_frames, width, height, n_freq, n_offsets, params, frames,
                         sensor, consts, bg, dout, steps=steps, flags=flags, n_sh=n_sh)
        table.append(dict(cfg, ms=round(ms, 4)))
    best = min(table, key=lambda c: c["ms"])
    result = dict(tile=tuple(best["tile"]), ppt=best["ppt"], mode=best["mode"], ms=best["ms"],
                  table=table)
    if cache_path:
        cache[key] = dict(result, tile=list(result["tile"]))
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return result
