"""Gradient checks of the CUDA path in double precision (the FP64
instantiation of every kernel): torch.autograd.gradcheck through the autograd
wrapper, and central finite differences per parameter group, on a
200-Gaussian 32x32 dynamic scene."""
import numpy as np
import pytest
import torch

from paper_2505_05356_gb300 import gftorf, scenes

pytestmark = pytest.mark.gpu

NAMES = ("means", "coeffs", "scales", "quats", "opacity", "amplitude", "delta")


def _setup(seed=0, n=200, W=32, H=32, frames=2):
    sc = scenes.make_scene("batch_300k", seed, n=n, width=W, height=H, frames=frames,
                           visible_min=0.7)
    r = gftorf.Renderer(sc.n, sc.frames, W, H, 1, 4, dtype=torch.float64,
                        max_instances=64 * n * frames)
    p = gftorf.params_from_scene(sc, dtype=torch.float64)
    fr, se, co = (gftorf.frames_from_scene(sc), gftorf.sensor_from_scene(sc),
                  gftorf.consts_from_scene(sc))
    bg = torch.as_tensor(sc.bg, device="cuda", dtype=torch.float64)
    return sc, r, p, fr, se, co, bg


def test_torch_gradcheck_fp64():
    sc, r, p, fr, se, co, bg = _setup()
    inputs = [p[k].clone().requires_grad_(True) for k in NAMES] + [bg.clone().requires_grad_(True)]

    def f(means, coeffs, scales, quats, opacity, amplitude, delta, bgi):
        return gftorf.RenderCToF.apply(r, fr, se, co, bgi, means, coeffs, scales, quats,
                                       opacity, amplitude, delta)

    assert torch.autograd.gradcheck(f, inputs, eps=1e-6, atol=1e-5, rtol=1e-4,
                                    fast_mode=True, nondet_tol=1e-12)
    code, _ = r.read_status()
    assert code == gftorf.OK


def _loss(r, p, fr, se, co, bg, w):
    r.preprocess(p, fr, se, co)
    return float((r.render_fwd(bg) * w).sum().item())


def test_central_differences_every_group_fp64():
    sc, r, p, fr, se, co, bg = _setup(seed=3)
    w = torch.randn((sc.frames, 5, sc.height, sc.width), dtype=torch.float64, device="cuda",
                    generator=torch.Generator(device="cuda").manual_seed(7))
    r.preprocess(p, fr, se, co)
    r.render_fwd(bg)
    g = r.render_bwd(p, bg, w)
    g = {k: v.cpu().numpy() for k, v in g.items()}
    base = _loss(r, p, fr, se, co, bg, w)
    rng = np.random.default_rng(4)
    checked = 0
    for name in NAMES:
        flat = p[name].view(-1)
        for i in rng.choice(flat.numel(), 25, replace=False):
            old = float(flat[i].item())
            h = 1e-6 * max(1.0, abs(old))
            flat[i] = old + h
            lp = _loss(r, p, fr, se, co, bg, w)
            flat[i] = old - h
            lm = _loss(r, p, fr, se, co, bg, w)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            if abs((lp - base) / h - (base - lm) / h) > 1e-3 * (abs(fd) + 1e-3):
                continue  # a discrete decision flips inside the step
            got = g[name].reshape(-1)[i]
            assert got == pytest.approx(fd, rel=1e-5, abs=1e-6 * (1 + abs(fd))), (name, i)
            checked += 1
    assert checked >= 120


def test_torch_gradcheck_sh_moved_camera_fp64():
    """SH reflectivity (degree 3) under a rotated, shifted camera: gradients of
    the SH coefficients and of the means through the view direction."""
    sc = scenes.make_scene("batch_300k", 8, n=150, width=32, height=32, frames=2,
                           visible_min=0.7, sh_degree=3, sh_std=0.1,
                           pose=((4.0, -6.0, 3.0), (0.1, -0.05, -0.2)))
    r = gftorf.Renderer(sc.n, sc.frames, 32, 32, 1, 4, dtype=torch.float64,
                        max_instances=64 * sc.n * sc.frames, n_sh=16)
    p = gftorf.params_from_scene(sc, dtype=torch.float64)
    fr, se, co = (gftorf.frames_from_scene(sc), gftorf.sensor_from_scene(sc),
                  gftorf.consts_from_scene(sc))
    bg = torch.as_tensor(sc.bg, device="cuda", dtype=torch.float64)
    names = ("means", "coeffs", "scales", "quats", "opacity", "delta", "sh")
    inputs = [p[k].clone().requires_grad_(True) for k in names]

    def f(means, coeffs, scales, quats, opacity, delta, sh):
        return gftorf.RenderCToF.apply(r, fr, se, co, bg, means, coeffs, scales, quats,
                                       opacity, None, delta, sh)

    assert torch.autograd.gradcheck(f, inputs, eps=1e-6, atol=1e-5, rtol=1e-4,
                                    fast_mode=True, nondet_tol=1e-12)
    assert r.read_status()[0] == gftorf.OK
