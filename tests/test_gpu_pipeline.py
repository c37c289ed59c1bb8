"""The host-streamed pipeline (copies of neighbouring steps overlapping the
compute) returns the same gradients as plain eager steps."""
import numpy as np
import pytest
import torch

from paper_2505_05356_gb300 import gftorf, scenes
from paper_2505_05356_gb300.pipeline import HostStream
from tests.gpu_helpers import grads_close

pytestmark = pytest.mark.gpu


def test_host_stream_matches_eager_steps():
    sc = scenes.make_scene("batch_300k", 17, n=4000, width=96, height=64, frames=3)
    r = gftorf.Renderer(sc.n, sc.frames, sc.width, sc.height, 1, 4, render_mode=1,
                        pixels_per_thread=4, tile=(16, 32))
    p = gftorf.params_from_scene(sc)
    fr, se, co = (gftorf.frames_from_scene(sc), gftorf.sensor_from_scene(sc),
                  gftorf.consts_from_scene(sc))
    bg = torch.as_tensor(sc.bg, device="cuda")
    dout = torch.as_tensor(scenes.random_dout(sc, 3), device="cuda")
    r.fit_capacity(p, fr, se, co, bg, headroom=1.5)
    r.preprocess(p, fr, se, co)
    r.render_fwd(bg)
    ref = r.render_bwd(p, bg, dout)
    torch.cuda.synchronize()
    ref = {k: v.double().cpu().numpy() for k, v in ref.items()}
    out = torch.empty((sc.frames, r.C, sc.height, sc.width), device="cuda")
    pnames = [k for k, v in p.items() if v is not None]
    host_in = {k: p[k].cpu().pin_memory() for k in pnames}
    host_in["bg"] = bg.cpu().pin_memory()
    host_in["dout"] = dout.cpu().pin_memory()
    template = r.alloc_grads(p, bg)
    host_out = {k: torch.zeros(v.shape, dtype=v.dtype, pin_memory=True)
                for k, v in template.items()}

    def make_set():
        ins = {k: torch.zeros_like(v, device="cuda") for k, v in host_in.items()}
        params = dict(p)
        params.update({k: ins[k] for k in pnames})
        return {"in": ins, "params": params,
                "out": {k: torch.empty_like(v) for k, v in template.items()}}

    def step(bufs):
        pr, gr, ins = bufs["params"], bufs["out"], bufs["in"]
        r.preprocess(pr, fr, se, co)
        r.bin()
        r.composite_fwd(ins["bg"], out)
        r.zero_grad_buffers(gr)
        r.composite_bwd(ins["bg"], ins["dout"], gr)
        r.preprocess_bwd(pr, gr)

    hs = HostStream(make_set, step)
    hs.run(host_in, host_out, 5)
    torch.cuda.synchronize()
    r.check()
    got = {k: v.double().numpy() for k, v in host_out.items()}
    for k, (nrm, elem) in grads_close(got, ref).items():
        assert nrm <= 1e-5, (k, nrm)
