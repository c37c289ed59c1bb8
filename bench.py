"""Benchmark: fwd+bwd raw C-ToF frames/s at 640x480 with 300k Gaussians.

One step = one batch of 16 timesteps of the 300k-Gaussian dynamic scene
(cubic trajectories, 30-100 % of the Gaussians visible per frame): deform +
project, bin + sort, composite (Eq. 4), then the backward (Eq. S3 re-walk,
chain rule to every Gaussian parameter), all in libgftorf's kernels,
replayed as one captured CUDA graph.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the baseline this path is compared with).
Multi-GPU (torchrun): every rank renders its own batch (independent
problems, no collective on the data path): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd raw C-ToF frames/sec at 640x480, 300k Gaussians; % HBM/FP32 roofline"


def metric_of(sc) -> str:
    """The metric's name for the workload actually run (the default workload
    gives METRIC)."""
    n = "%dk" % (sc.n // 1000) if sc.n % 1000 == 0 else str(sc.n)
    return ("fwd+bwd raw C-ToF frames/sec at {}x{}, {} Gaussians; % HBM/FP32 roofline"
            .format(sc.width, sc.height, n))
UNIT = "frames/s"
WORKLOAD = "batch_300k"

# Algorithmic work per unit: FP32 lane operations per
# evaluated (pixel, Gaussian) pair of the compositing kernels, and bytes per
# Gaussian-frame / per instance of the memory-bound stages.  An evaluated pair
# is one the kernels actually walk: per pixel, the records of its tile's list
# that can reach its warp's pixels, up to and including the one that stops
# it (the forward's counting instantiation counts them); the tile list's
# candidates before the per-warp masks (a count that grows with the tile's
# size) are reported beside it.
OPS_PER_PAIR_FWD = 20
OPS_PER_PAIR_BWD = 60


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return p, "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _overrides(args):
    """Smaller variants of the workload (profiling captures only)."""
    o = {}
    for ch in (args.extra_channels or "").split(","):
        if ch in ("phasor", "depth"):
            o[ch] = True
    if args.frames:
        o["frames"] = args.frames
    if args.n:
        o["n"] = args.n
    if args.sh_degree >= 0:
        o["sh_degree"] = args.sh_degree
    if args.async_capture:
        o["async_capture"] = True
    return o


KERNEL_OF_STAGE = {"composite_bwd": "render_bwd_kernel", "composite_fwd": "render_fwd_kernel"}


def _traffic(stage, frames):
    """DRAM bytes per launch of the stage's kernel from the committed ncu
    capture (profiles/traffic.json), scaled to `frames` when the capture ran
    another batch size; None when the kernel's source changed since the
    capture or none exists."""
    import hashlib
    kern = KERNEL_OF_STAGE.get(stage)
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if kern is None or not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f).get(kern)
    src = os.path.join(ROOT, "paper_2505_05356_gb300", "csrc", "render_impl.cuh")
    with open(src, "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()[:16]
    if not rec or rec.get("source_sha256_16") != h:
        return None
    return int(rec["dram_bytes_per_launch"] * frames / rec["frames_in_capture"])


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest value of x over all ranks (the job's time is its slowest
    rank's); identity on one process."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
# the other full-size workloads, measured after the headline one and reported
# as extra keys of the same line (100k Gaussians at 640x480, one frame per
# step; 500k Gaussians at 640x576 with 30 and 80 MHz, 8 frames per step)
EXTRA_WORKLOADS = ("dynamic_100k", "twofreq_500k")


def workload_config(sc, name, args) -> dict:
    """The workload a line measures (shared by both arms, no launch choices)."""
    nF, nP = len(sc.sensor.freqs_hz), len(sc.sensor.offsets_rad)
    vis = ", 30-100%% visible per frame" if name in ("batch_300k", "twofreq_500k") else ""
    return {"workload": "%s: %d dynamic Gaussians (cubic trajectories), %dx%d, "
                        "%d timesteps per batch, %s MHz x %d offsets + ambient%s" % (
                            name, sc.n, sc.width, sc.height, sc.frames,
                            "+".join("%g" % (f / 1e6) for f in sc.sensor.freqs_hz), nP, vis),
            "frames_per_step": sc.frames, "channels": sc.n_channels,
            "reflectivity": ("SH degree %d" % args.sh_degree
                             if args.sh_degree >= 0 else "scalar"),
            "capture": ("asynchronous (1 offset per frame, Eq. 7 motion)"
                        if args.async_capture else "synchronous quartets")}


def measure(sc, args, steps, warmup, world=1, seed=0, autotune=True, want_e2e=False,
            want_plain=False, alu=None):
    """Time the batched, graph-captured fwd+bwd step of scene `sc`: the step
    rate, per-stage CUDA-event times, each stage against its roofline, and
    optionally the end-to-end rate through the public API from pinned host
    memory and the same work as per-frame plain launches."""
    import torch
    import torch.distributed as dist

    from paper_2505_05356_gb300 import gftorf, scenes

    B, N, W, H = sc.frames, sc.n, sc.width, sc.height
    nF, nP = len(sc.sensor.freqs_hz), len(sc.sensor.offsets_rad)
    xflags = gftorf.flags_from_scene(sc)
    p = gftorf.params_from_scene(sc)
    fr = gftorf.frames_from_scene(sc)
    se = gftorf.sensor_from_scene(sc)
    co = gftorf.consts_from_scene(sc)
    bg = torch.as_tensor(sc.bg, device="cuda")
    dout = torch.as_tensor(scenes.random_dout(sc, 100 + seed), device="cuda")
    tile = tuple(int(v) for v in args.tile.split("x"))
    ppt, mode = args.ppt, args.mode
    tuned = None
    if autotune:
        from paper_2505_05356_gb300 import autotune as at
        tuned = at.autotune(N, B, W, H, nF, nP, p, fr, se, co, bg, dout, steps=2,
                            flags=xflags, n_sh=sc.n_sh)
        tile, ppt, mode = tuned["tile"], tuned["ppt"], tuned["mode"]
    r = gftorf.Renderer(N, B, W, H, nF, nP, tile=tile, render_mode=mode,
                        pixels_per_thread=ppt, flags=xflags, n_sh=sc.n_sh)
    r.fit_capacity(p, fr, se, co, bg)
    out = torch.empty((B, r.C, H, W), device="cuda")
    grads = r.alloc_grads(p, bg)

    def step():
        r.preprocess(p, fr, se, co)
        r.bin()
        r.composite_fwd(bg, out)
        r.zero_grad_buffers(grads)
        r.composite_bwd(bg, dout, grads)
        r.preprocess_bwd(p, grads)

    # eager warm-up + kernels per step
    step()
    torch.cuda.synchronize()
    r.check()
    k0 = gftorf.kernel_launches()
    step()
    torch.cuda.synchronize()
    kernels_per_step = gftorf.kernel_launches() - k0

    use_graph = not args.no_graph
    if use_graph:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            step()
        torch.cuda.current_stream().wait_stream(s)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        run = graph.replay
    else:
        run = step
    for _ in range(warmup):
        run()
    torch.cuda.synchronize()

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        run()
    e1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    code, count = r.read_status()
    if code != gftorf.OK:
        raise RuntimeError("device status %s" % gftorf.STATUS.get(code))
    ms = max_over_ranks(ms, world, "cuda")
    res = {"ms_per_step": ms / steps, "value": world * B * steps / (ms / 1e3),
           "kernels_per_step": int(kernels_per_step), "tile": tile, "ppt": ppt, "mode": mode,
           "tuned": tuned, "ws_bytes": r.ws_bytes, "C": r.C, "use_graph": use_graph}

    # --- per-stage timing (same stream, CUDA events, eager) ---
    stages = ["preprocess", "bin", "composite_fwd", "zero_grad_buffers", "composite_bwd",
              "preprocess_bwd"]
    calls = [lambda: r.preprocess(p, fr, se, co), r.bin, lambda: r.composite_fwd(bg, out),
             lambda: r.zero_grad_buffers(grads), lambda: r.composite_bwd(bg, dout, grads),
             lambda: r.preprocess_bwd(p, grads)]
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)]
          for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        ev[k][0].record()
        for i, c in enumerate(calls):
            c()
            ev[k][i + 1].record()
    torch.cuda.synchronize()
    stage_ms = {s_: sum(ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(steps)) / steps
                for i, s_ in enumerate(stages)}

    # --- algorithmic work of this batch: evaluated (pixel, Gaussian) pairs
    # counted by the forward's counting instantiation on the same inputs ---
    rc = gftorf.Renderer(N, B, W, H, nF, nP, tile=tile, render_mode=mode,
                         pixels_per_thread=ppt, flags=gftorf.FLAG_COUNT_PAIRS | xflags,
                         max_instances=r.capacity, n_sh=sc.n_sh)
    rc.preprocess(p, fr, se, co)
    rc.render_fwd(bg)
    instances, pairs, pairs_warp = rc.counters(with_warp=True)
    del rc
    torch.cuda.empty_cache()
    peaks, peak_kind = _peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    if alu is not None:
        alu_peak = alu["ffma"] / 1e9  # G FP32 lane-ops/s, measured in this run
        alu_src = "measured FFMA loop (gftorf_probe_throughput, this run)"
    else:
        n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        alu_peak = n_sm * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e9
        alu_src = "nominal: SMs x 128 FP32 lanes x max SM clock"
    vis = B * N  # upper bound of Gaussian-frames
    work = {
        "composite_bwd": ("alu", pairs_warp * OPS_PER_PAIR_BWD / 1e9, "Gop/s", alu_peak, alu_src),
        "composite_fwd": ("alu", pairs_warp * OPS_PER_PAIR_FWD / 1e9, "Gop/s", alu_peak, alu_src),
        # read 84 B of parameters + write a 48 B record, 8 B rect, 4 B key
        # (+ 4 B per SH coefficient read with the parameters)
        "preprocess": ("hbm", vis * (84 + 60 + 4 * sc.n_sh) / 1e9, "GB/s", hbm_peak, peak_kind),
        # instance values written once; depth keys 4 passes x 16 B
        "bin": ("hbm", (instances * 4 + vis * 16 * 4) / 1e9, "GB/s", hbm_peak, peak_kind),
        "preprocess_bwd": ("hbm", (vis * (84 + 36 + 12) + N * 8 * sc.n_sh) / 1e9, "GB/s",
                           hbm_peak, peak_kind),
        "zero_grad_buffers": ("hbm", vis * 36 / 1e9, "GB/s", hbm_peak, peak_kind),
    }
    stage_rows = {}
    for s_ in stages:
        b_, a_, u_, pk_, src_ = work[s_]
        ach = a_ / (stage_ms[s_] / 1e3) if stage_ms[s_] > 0 else 0.0
        row = {"ms": round(stage_ms[s_], 4), "bound": b_, "achieved": round(ach, 1),
               "unit": u_, "peak": round(pk_, 1), "frac": round(ach / pk_, 4)}
        if b_ == "alu":
            # the same per tile-list candidate pair (before the per-warp masks)
            row["frac_per_list_pair"] = round(ach * pairs / max(pairs_warp, 1) / pk_, 4)
        if b_ == "alu" and alu is not None:
            # one ex2 per evaluated pair: the multi-function unit's share
            ex2 = pairs_warp / (stage_ms[s_] / 1e3) / 1e9
            row["mufu"] = {"achieved": round(ex2, 1), "peak": round(alu["ex2"] / 1e9, 1),
                           "unit": "G ex2/s", "frac": round(ex2 / (alu["ex2"] / 1e9), 4)}
        stage_rows[s_] = row
    dom = max(stage_ms, key=stage_ms.get)
    b_, a_, u_, pk_, src_ = work[dom]
    achieved = a_ / (stage_ms[dom] / 1e3)
    roofline = {"kernel": dom, "bound": b_, "achieved": round(achieved, 2),
                "peak": round(pk_, 2), "unit": u_, "frac": round(achieved / pk_, 4),
                "traffic": _traffic(dom, B), "peak_source": src_}
    if b_ == "alu":
        roofline["work"] = ("%d FP32 lane-ops per evaluated (pixel, Gaussian) pair x %d pairs "
                            "(after the per-warp record masks)"
                            % (OPS_PER_PAIR_BWD if dom == "composite_bwd" else OPS_PER_PAIR_FWD,
                               pairs_warp))
        roofline["frac_per_list_pair"] = stage_rows[dom]["frac_per_list_pair"]
    if "mufu" in stage_rows[dom]:
        roofline["mufu"] = stage_rows[dom]["mufu"]
    res.update(stage_rows=stage_rows, roofline=roofline, instances=instances, pairs=pairs,
               pairs_warp=pairs_warp)

    # --- end to end through the public API with host buffers ---
    if want_e2e:
        # end to end from pinned host memory: every step copies its inputs in
        # and its gradients out; the copies of neighbouring steps overlap the
        # compute (two buffer sets, two graphs, copy streams; pipeline.py)
        from paper_2505_05356_gb300.pipeline import HostStream

        pnames = [k for k, v in p.items() if v is not None]
        host_in = {k: p[k].cpu().pin_memory() for k in pnames}
        host_in["bg"] = bg.cpu().pin_memory()
        host_in["dout"] = dout.cpu().pin_memory()
        host_out = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
                    for k, v in grads.items()}
        h2d = sum(t.numel() * t.element_size() for t in host_in.values())
        d2h = sum(t.numel() * t.element_size() for t in host_out.values())

        def make_set():
            ins = {k: torch.empty_like(v, device="cuda") for k, v in host_in.items()}
            for k, v in host_in.items():
                ins[k].copy_(v)
            params = dict(p)
            params.update({k: ins[k] for k in pnames})
            return {"in": ins, "params": params,
                    "out": {k: torch.empty_like(v) for k, v in grads.items()}}

        def set_step(bufs):
            pr, gr, ins = bufs["params"], bufs["out"], bufs["in"]
            r.preprocess(pr, fr, se, co)
            r.bin()
            r.composite_fwd(ins["bg"], out)
            r.zero_grad_buffers(gr)
            r.composite_bwd(ins["bg"], ins["dout"], gr)
            r.preprocess_bwd(pr, gr)

        hs = HostStream(make_set, set_step)
        hs.run(host_in, host_out, 2)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        hs.run(host_in, host_out, steps, start=a0)
        a1.record()
        torch.cuda.synchronize()
        ems = max_over_ranks(a0.elapsed_time(a1), world, "cuda")
        res["e2e"] = {"value": round(world * B * steps / (ems / 1e3), 2), "unit": UNIT,
                      "pipelined": "host->device of step i+1 and device->host of step i-1 "
                                   "overlap step i (two buffer sets, two CUDA graphs, copy "
                                   "streams)",
                      "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # --- per-frame plain launches (no batching, no graph), same work ---
    if want_plain:
        r1 = gftorf.Renderer(N, 1, W, H, nF, nP, tile=tile, render_mode=0,
                             pixels_per_thread=ppt, flags=xflags, n_sh=sc.n_sh,
                             max_instances=max(1024, int(r.capacity / B * 1.6)))
        gacc = {k: torch.zeros_like(v) for k, v in grads.items() if k not in ("bg", "delta")}
        p1s = []
        for b in range(B):
            p1 = dict(p)
            p1["delta"] = p["delta"][b:b + 1].contiguous() if p["delta"] is not None else None
            p1s.append(p1)
        bgs = [bg[b:b + 1].contiguous() for b in range(B)]
        douts = [dout[b:b + 1].contiguous() for b in range(B)]
        out1 = torch.empty((1,) + tuple(out.shape[1:]), device="cuda")
        g1 = r1.alloc_grads(p1s[0], bgs[0])

        def plain_step():
            for v in gacc.values():
                v.zero_()
            for b in range(B):
                r1.preprocess(p1s[b], [fr[b]], se, co)
                r1.render_fwd(bgs[b], out1)
                r1.render_bwd(p1s[b], bgs[b], douts[b], grads=g1)
                for k, v in gacc.items():
                    v.add_(g1[k])

        for _ in range(max(2, warmup)):
            plain_step()
        torch.cuda.synchronize()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record()
        for _ in range(steps):
            plain_step()
        q1.record()
        torch.cuda.synchronize()
        pms = q0.elapsed_time(q1) / steps
        code1, _ = r1.read_status()
        res["plain"] = {"value": round(B / (pms / 1e3), 2), "unit": UNIT,
                        "ms_per_step": round(pms, 3), "status": gftorf.STATUS.get(code1)}
        del r1
    del r, out, grads
    torch.cuda.empty_cache()
    return res


def launch_config(m, args) -> dict:
    """The launch choices a measurement ran with (autotuned unless asked)."""
    return {"tile": "%dx%d" % tuple(m["tile"]), "pixels_per_thread": m["ppt"],
            "render_mode": "persistent" if m["mode"] == 1 else "grid",
            "autotuned": m["tuned"] is not None, "cuda_graph": m["use_graph"],
            "kernels_per_step": m["kernels_per_step"]}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2505_05356_gb300 import gftorf, scenes

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    sc = scenes.make_scene(args.workload, seed=rank, **_overrides(args))
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    # the compositing kernels' denominators, measured on this GPU in this run
    alu = gftorf.measure_alu_peaks()
    m = measure(sc, args, args.steps, args.warmup, world=world, seed=rank,
                autotune=args.autotune, want_e2e=not args.skip_e2e,
                want_plain=not args.skip_plain and rank == 0, alu=alu)
    clk = clocks.stop()

    extras = {}
    if rank == 0 and not args.skip_extra and not _overrides(args):
        for name in EXTRA_WORKLOADS:
            if name == args.workload:
                continue
            esc = scenes.make_scene(name, seed=0)
            em = measure(esc, args, min(args.steps, 10), max(3, min(args.warmup, 5)),
                         autotune=args.autotune, alu=alu)
            extras[name] = {"metric": metric_of(esc), "value": round(em["value"], 2),
                            "unit": UNIT, "ms_per_step": round(em["ms_per_step"], 4),
                            "config": workload_config(esc, name, args),
                            "launch": launch_config(em, args),
                            "roofline": em["roofline"], "stages": em["stage_rows"],
                            "instances_per_step": em["instances"],
                            "evaluated_pairs_per_step": em["pairs_warp"],
                            "list_pairs_per_step": em["pairs"],
                            "autotune": None if em["tuned"] is None else em["tuned"]["table"]}
    if world > 1:
        dist.barrier()

    fitres = None
    if not args.skip_fit and rank == 0:
        fitres = fit_loop_bench(args, m["tile"], m["ppt"], m["mode"])
    mlpres = None
    if not args.skip_mlp and rank == 0:
        mlpres = mlp_bench(args, frames=tuple(int(v) for v in args.mlp_frames.split(",") if v))

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        cpu = cpu_baseline(sc, args.cpu_seconds)

    if rank == 0:
        launch = launch_config(m, args)
        launch.update({"parallelism": "replicas" if world > 1 else "1 GPU",
                       "l2": "inputs larger than L2 (%.0f MB workspace per step)"
                             % (m["ws_bytes"] / 1e6),
                       "instances_per_step": m["instances"],
                       "evaluated_pairs_per_step": m["pairs_warp"],
                       "list_pairs_per_step": m["pairs"]})
        line = {
            "metric": metric_of(sc), "value": round(m["value"], 2), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(m["ms_per_step"], 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded; shaped like the paper's C-ToF scenes)",
            "config": workload_config(sc, args.workload, args),
            "launch": launch,
            "gpu_launches": int(m["kernels_per_step"] * args.steps),
            "kernels_per_step": int(m["kernels_per_step"]),
            "roofline": m["roofline"],
            "alu_peaks": {"ffma_g_lane_ops_s": round(alu["ffma"] / 1e9, 1),
                          "ex2_g_lane_ops_s": round(alu["ex2"] / 1e9, 1),
                          "how": "gftorf_probe_throughput: 8 x 256-thread CTAs per SM, 8 "
                                 "independent chains per thread, best of 5 launches, CUDA "
                                 "events; clocks as in 'clocks'"},
            "stages": m["stage_rows"],
            "e2e": m.get("e2e"),
            "per_frame_plain": m.get("plain"),
            "workloads": extras or None,
            "optimization_loop": fitres,
            "deformation_mlp": mlpres,
            "cpu_baseline": cpu,
            "clocks": clk,
            "autotune": None if m["tuned"] is None else m["tuned"]["table"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# optimisation loop: iterations/s of the whole fit step, batched + graph vs
# plain per-frame launches (same frames, same work)
# ---------------------------------------------------------------------------
def fit_loop_bench(args, tile, ppt, mode):
    import torch

    from paper_2505_05356_gb300 import fit, gftorf, scenes

    gt, init = scenes.make_fit_scenes(seed=4)
    B, W, H = gt.frames, gt.width, gt.height
    fr, se, co = (gftorf.frames_from_scene(gt), gftorf.sensor_from_scene(gt),
                  gftorf.consts_from_scene(gt))
    # the captured raw frames: the ground-truth scene rendered once
    rg = gftorf.Renderer(gt.n, B, W, H, 1, 4, tile=tile, render_mode=mode, pixels_per_thread=ppt)
    pg = gftorf.params_from_scene(gt)
    zero_bg = torch.zeros((B, rg.C), device="cuda")
    rg.fit_capacity(pg, fr, se, co, zero_bg)
    rg.preprocess(pg, fr, se, co)
    targets = rg.render_fwd(zero_bg).clone()
    rg.check()
    del rg, pg
    torch.cuda.empty_cache()

    p = gftorf.params_from_scene(init)
    p0 = {k: v.clone() for k, v in p.items() if v is not None}
    loop = fit.FitLoop(p, fr, se, co, targets, tile=tile, pixels_per_thread=ppt,
                       render_mode=mode, seed=11)
    loop.run(1)
    torch.cuda.synchronize()
    k0 = gftorf.kernel_launches()
    loop.run(1)
    torch.cuda.synchronize()
    kernels_per_it = gftorf.kernel_launches() - k0
    loop.capture()
    loop.run(max(3, args.warmup))
    torch.cuda.synchronize()
    loss_start = loop.loss()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    loop.run(args.fit_iters)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.fit_iters
    loop.check()
    loss_end = loop.loss()
    its = loop.step

    # plain: the same iteration as per-frame launches, no graph
    for k, v in p0.items():
        p[k].copy_(v)
    r1 = gftorf.Renderer(init.n, 1, W, H, 1, 4, tile=tile, render_mode=0, pixels_per_thread=ppt,
                         max_instances=max(1024, int(loop.r.capacity / B * 1.6)))
    st = gftorf.new_train_state()
    bg = torch.zeros((B, r1.C), device="cuda")
    gacc = {k: torch.zeros_like(p[k]) for k in fit.LEARNING_RATES}
    g1 = r1.alloc_grads(p, bg[0:1], want=list(fit.LEARNING_RATES))
    opt = gftorf.Adam(p, fit.LEARNING_RATES, fit.BOUNDS)
    out1 = torch.empty((1, r1.C, H, W), device="cuda")
    d1 = torch.empty_like(out1)
    tg = [targets[b:b + 1] for b in range(B)]
    bgs = [bg[b:b + 1] for b in range(B)]

    def plain_iteration():
        gftorf.train_begin(st, bg, 11)
        for v in gacc.values():
            v.zero_()
        for b in range(B):
            r1.preprocess(p, [fr[b]], se, co)
            r1.render_fwd(bgs[b], out1)
            gftorf.l2_loss(r1, out1, tg[b], d1, st)
            r1.render_bwd(p, bgs[b], d1, grads=g1)
            for k, v in gacc.items():
                v.add_(g1[k])
        opt.step(gacc, st)

    n_plain = max(2, min(5, args.fit_iters))
    plain_iteration()
    torch.cuda.synchronize()
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    q0.record()
    for _ in range(n_plain):
        plain_iteration()
    q1.record()
    torch.cuda.synchronize()
    pms = q0.elapsed_time(q1) / n_plain
    code1, _ = r1.read_status()
    return {"workload": "fit of %d Gaussians (random init in the frustum, reflectivity 0.1) to "
                        "%d raw frames %dx%d of a %d-Gaussian scene (backdrop + 0.8 m rod "
                        "swinging at 2 m/s peak); per iteration: random bg, fwd, L2 loss on "
                        "the raw samples, bwd, fused Adam over 6 groups"
                        % (init.n, B, W, H, gt.n),
            "frames_per_iteration": B,
            "graph_it_per_s": round(1e3 / ms, 2), "graph_ms_per_it": round(ms, 3),
            "plain_it_per_s": round(1e3 / pms, 2), "plain_ms_per_it": round(pms, 3),
            "speedup": round(pms / ms, 2), "kernels_per_iteration": int(kernels_per_it),
            "iterations_run": its, "loss_after_warmup": loss_start, "loss_last": loss_end,
            "plain_status": gftorf.STATUS.get(code1)}


# ---------------------------------------------------------------------------
# deformation MLP on the tensor cores: fwd + bwd of all Gaussians at one
# timestep (one fitting iteration's MLP work) and at the batch's 16 timesteps
# ---------------------------------------------------------------------------
MLP_FLOPS_PER_ROW = 2.0 * (84 * 256 + 7 * 256 * 256 + 3 * 256)  # forward; backward 2x


def mlp_bench(args, n=300_000, frames=(1, 16)):
    import torch

    from paper_2505_05356_gb300 import mlp, scenes

    peaks, _ = _peaks()
    peak = peaks.get("bf16_tflops", 1900.0)
    theta = torch.as_tensor(scenes.init_mlp_params(0, head_std=0.05), device="cuda")
    rng = np.random.default_rng(0)
    mu = torch.as_tensor(rng.uniform(-2.0, 4.0, (n, 3)).astype(np.float32), device="cuda")
    out = {}
    for B in frames:
        net = mlp.DeformationMLP(n, B, 1.0 / mlp.unambiguous_range(30e6))
        times = list(np.linspace(0.0, 1.0, B))
        dd = torch.randn((B, n, 3), device="cuda")
        for _ in range(2):
            net.forward(theta, mu, times)
            net.backward(theta, mu, times, dd)
        torch.cuda.synchronize()
        k = args.mlp_iters if args.mlp_iters else (5 if B == 1 else 2)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        tf = tb = 0.0
        for _ in range(k):
            ev[0].record()
            net.forward(theta, mu, times)
            ev[1].record()
            net.backward(theta, mu, times, dd)
            ev[2].record()
            torch.cuda.synchronize()
            tf += ev[0].elapsed_time(ev[1]) / k
            tb += ev[1].elapsed_time(ev[2]) / k
        net.check()
        # inference forward (fused kernel, activations on chip)
        net.infer(theta, mu, times)
        torch.cuda.synchronize()
        ti = 0.0
        for _ in range(k):
            ev[0].record()
            net.infer(theta, mu, times)
            ev[1].record()
            torch.cuda.synchronize()
            ti += ev[0].elapsed_time(ev[1]) / k
        net.check()
        rows = n * B
        tfi = MLP_FLOPS_PER_ROW * rows / (ti / 1e3) / 1e12
        flops = 3.0 * MLP_FLOPS_PER_ROW * rows
        tfl = flops / ((tf + tb) / 1e3) / 1e12
        out["rows_%d" % rows] = {
            "frames": B, "fwd_ms": round(tf, 3), "bwd_ms": round(tb, 3),
            "tflops": round(tfl, 1),
            "infer_fused": {"ms": round(ti, 3), "tflops": round(tfi, 1),
                            "frac": round(tfi / peak, 4)},
            "roofline": {"bound": "tensor", "achieved": round(tfl, 1), "peak": peak,
                         "unit": "TFLOP/s", "frac": round(tfl / peak, 4),
                         "peak_source": "measured bf16 (burst)"}}
        del net
        torch.cuda.empty_cache()
    out["network"] = ("positional encoding (10 freq) 84 -> 8 x 256 ReLU -> 3, BF16 tcgen05 "
                      "GEMMs with FP32 accumulation; algorithmic FLOPs 3 x %.0f per row "
                      "(forward + weight and input gradients)" % MLP_FLOPS_PER_ROW)
    return out


# ---------------------------------------------------------------------------
# CPU oracle timing (baseline; bounded sample of the same workload)
# ---------------------------------------------------------------------------
def oracle_sample(sc, n_pix, frame=0, seed=5):
    """Time the FP64 oracle's fwd+bwd on about n_pix pixels of one frame --
    all pixels of randomly chosen tiles, so that the per-tile work (the
    backward's candidate lists) and the per-pixel work scale alike -- and
    extrapolate to frames/s.  Returns (frames_per_s, seconds_spent, detail)."""
    from oracle import oracle as ora
    from paper_2505_05356_gb300 import scenes

    one = scenes.Scene(sc.means, sc.coeffs, sc.scales, sc.quats, sc.opacity, sc.amplitude,
                       sc.times[frame:frame + 1], sc.cameras[frame:frame + 1],
                       None if sc.delta is None else sc.delta[frame:frame + 1],
                       sc.sensor, sc.consts, sc.bg[frame:frame + 1], sc.sh)
    HW = sc.width * sc.height
    rng = np.random.default_rng(seed)
    TW, TH = sc.consts.tile_w, sc.consts.tile_h
    tx_n, ty_n = -(-sc.width // TW), -(-sc.height // TH)
    k = int(min(tx_n * ty_n, max(1, round(n_pix * tx_n * ty_n / HW))))  # tiles, on average
    tiles = rng.choice(tx_n * ty_n, k, replace=False)
    xs, ys = np.meshgrid(np.arange(TW), np.arange(TH))
    pix = np.concatenate([np.stack([xs.ravel() + (t % tx_n) * TW, ys.ravel() + (t // tx_n) * TH], 1)
                          for t in tiles])
    pix = pix[(pix[:, 0] < sc.width) & (pix[:, 1] < sc.height)].astype(np.int32)
    n_pix = len(pix)
    P = ora.Params(one)
    t0 = time.perf_counter()
    sp = ora.project(one, 0, ora.EPS_NONE, P)
    t1 = time.perf_counter()
    ora.render_pixels(one, 0, pix, sp)
    t2 = time.perf_counter()
    dout = np.zeros((sc.n_channels, sc.height, sc.width))
    dout[:, pix[:, 1], pix[:, 0]] = 1.0
    nf = 2 * len(sc.sensor.freqs_hz) + 1
    g2d = np.zeros((sc.n, 7 + nf))
    lib = ora.lib()
    fr, se, co = ora.pack_frame(one, 0), ora.pack_sensor(one), ora.pack_consts(one)
    bg0 = np.ascontiguousarray(one.bg[0], np.float64)
    lib.ora_backward_2d(sc.n, ora._p(sp), ora._p(fr), ora._p(se), ora._p(co), ora._p(bg0),
                        ora._p(dout), ora._p(g2d), None)
    t3 = time.perf_counter()
    # the 2D backward's per-frame part (its pass over every pixel for the
    # nonzero dL/dQ) is not scaled with the sample: timed with no pixel set
    g2d0 = np.zeros_like(g2d)
    u0 = time.perf_counter()
    lib.ora_backward_2d(sc.n, ora._p(sp), ora._p(fr), ora._p(se), ora._p(co), ora._p(bg0),
                        ora._p(np.zeros_like(dout)), ora._p(g2d0), None)
    bwd_fixed = min(time.perf_counter() - u0, t3 - t2)
    t3c = time.perf_counter()
    grads = np.zeros((sc.n, ora.NPARAM))
    lib.ora_backward_params(sc.n, ora._p(P.means), ora._p(P.coeffs), ora._p(P.scales),
                            ora._p(P.quats), ora._p(P.opacity), ora._p(P.amplitude),
                            ora._p(P.delta_of(0)), ora._p(P.sh), ora._p(fr), ora._p(se),
                            ora._p(co),
                            ora._p(sp), ora._p(g2d), ora._p(grads))
    t4 = time.perf_counter()
    chain = t4 - t3c
    touched = int(np.count_nonzero(np.any(g2d != 0, axis=1)))
    visible = int(np.count_nonzero(sp[:, ora.SP["VIS"]]))
    per_frame = ((t1 - t0) + ((t2 - t1) + (t3 - t2 - bwd_fixed)) * HW / n_pix + bwd_fixed +
                 chain * (visible / max(touched, 1)))
    detail = dict(project_s=t1 - t0, fwd_pixels_s=t2 - t1, bwd_pixels_s=t3 - t2,
                  bwd_frame_s=bwd_fixed, chain_s=chain, touched=touched, visible=visible,
                  pixels=n_pix, tiles=k)
    return 1.0 / per_frame, (t4 - t0) - bwd_fixed, detail


def _calibrate(sc, seconds):
    """Pixels per sample so that one oracle sample takes about `seconds`: a
    64-pixel probe, then a probe at a quarter of the target, which sets the
    per-pixel cost free of fixed overheads."""
    n = 64
    for frac in (0.25, 1.0):
        _, spent, det = oracle_sample(sc, n)
        per_px = max(det["fwd_pixels_s"] + det["bwd_pixels_s"], 1e-6) / det["pixels"]
        fixed = det["project_s"] + det["chain_s"]
        n = int(min(sc.width * sc.height, max(64, (frac * seconds - fixed) / per_px)))
    return n


def cpu_baseline(sc, seconds):
    from oracle import oracle as ora
    n_pix = _calibrate(sc, seconds)
    threads = ora.num_threads()
    fps, spent, det = oracle_sample(sc, n_pix, seed=6)
    # the same on one thread, on a proportionally smaller sample
    n1 = max(64, n_pix // (8 * max(threads, 1)))
    ora.set_threads(1)
    try:
        fps1, spent1, det1 = oracle_sample(sc, n1, seed=7)
    finally:
        ora.set_threads(threads)
    return {"value": round(fps, 6), "unit": UNIT, "cores": threads, "nproc": os.cpu_count(),
            "kind": "oracle",
            "sample": "frame 0 of the batch: projection of all %d Gaussians + fwd/bwd of the "
                      "%d pixels of %d random tiles (of %d pixels) + chain rule of the %d "
                      "touched Gaussians, extrapolated to a full frame (%.1f s of CPU work)"
                      % (sc.n, det["pixels"], det["tiles"], sc.width * sc.height,
                         det["touched"], spent),
            "single_thread": {"value": round(fps1, 6), "unit": UNIT,
                              "sample": "the same with the %d pixels of %d tile(s) on one "
                                        "thread (%.1f s)"
                                        % (det1["pixels"], det1["tiles"], spent1)}}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import oracle as ora
    from paper_2505_05356_gb300 import scenes

    sc = scenes.make_scene(args.workload, seed=0, **_overrides(args))
    budget = max(5.0, args.cpu_seconds / max(args.steps + args.warmup, 1))
    n_pix = _calibrate(sc, budget)
    for w in range(args.warmup):
        oracle_sample(sc, max(16, n_pix // 8), frame=w % sc.frames, seed=w)
    rates, total = [], 0.0
    for k in range(args.steps):
        fps, spent, det = oracle_sample(sc, n_pix, frame=k % sc.frames, seed=100 + k)
        rates.append(fps)
        total += spent
    value = len(rates) / sum(1.0 / x for x in rates)  # frames per second over the steps
    line = {
        "impl": "reference", "metric": metric_of(sc), "value": round(value, 6), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * sc.frames / value, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded; shaped like the paper's C-ToF scenes)",
        "config": workload_config(sc, args.workload, args),
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": ora.num_threads(),
                         "nproc": os.cpu_count(), "kind": "oracle",
                         "sample": "per step one frame: projection of all Gaussians + fwd/bwd of "
                                   "the pixels of random tiles (about %d pixels) + chain rule of "
                                   "the touched Gaussians, extrapolated to the full frame"
                                   % n_pix},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--tile", default="16x16")
    ap.add_argument("--mode", type=int, default=0, help="0 grid, 1 persistent")
    ap.add_argument("--ppt", type=int, default=4, help="pixels per compositing thread")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="use --tile/--ppt/--mode instead of timing every configuration")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-extra", action="store_true",
                    help="skip the other full-size workloads (100k at 640x480; 500k, 2 freq)")
    ap.add_argument("--skip-fit", action="store_true",
                    help="skip the optimisation-loop measurement (iterations/s)")
    ap.add_argument("--fit-iters", type=int, default=20)
    ap.add_argument("--skip-mlp", action="store_true",
                    help="skip the deformation-MLP measurement (tensor cores)")
    ap.add_argument("--mlp-only", action="store_true",
                    help="run only the deformation-MLP measurement (profiling)")
    ap.add_argument("--mlp-frames", default="1,16",
                    help="timesteps of 300k Gaussians per MLP measurement, comma list")
    ap.add_argument("--mlp-iters", type=int, default=0,
                    help="timed MLP forward+backward passes (0: 5 at one frame, else 2)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--frames", type=int, default=0, help="override frames per batch")
    ap.add_argument("--n", type=int, default=0, help="override the Gaussian count")
    ap.add_argument("--extra-channels", default="",
                    help="comma list of extra outputs: phasor (Eq. 3), depth (Eq. 5)")
    ap.add_argument("--async-capture", action="store_true",
                    help="asynchronous raw capture: one phase offset per frame, Eq. 7 "
                         "piecewise-linear motion between quartets")
    ap.add_argument("--sh-degree", type=int, default=-1,
                    help="view-dependent reflectivity from SH of this degree (0-3); "
                         "default: scalar reflectivity")
    args = ap.parse_args()
    if args.mlp_only:
        import torch
        torch.cuda.set_device(0)
        frames = tuple(int(v) for v in args.mlp_frames.split(",") if v)
        print(json.dumps({"deformation_mlp": mlp_bench(args, frames=frames)}), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
