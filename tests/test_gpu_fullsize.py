"""Parity at full size -- the benchmark's workload (300k dynamic Gaussians,
640x480, 16 timesteps) in the launch configurations bench.py times, and the
other full-size workloads (100k Gaussians at 640x480; 500k Gaussians at
640x576 with two modulation frequencies, 8 timesteps) -- on whole tiles
sampled at random (every pixel of 16 tiles per frame: the kernels' long tile
lists, staging rounds and block exits at full density), which the oracle
renders tile by tile, and gradients of a loss that only sees those pixels
(exactly computable by the oracle).  Pixels whose single-precision result may
take a near-threshold decision the other way are compared with the oracle's
walk that took it the same way."""
import numpy as np
import pytest
import torch

from oracle import oracle as ora
from paper_2505_05356_gb300 import gftorf, scenes
from tests.gpu_helpers import absent_groups, grads_close, match_alternatives

pytestmark = pytest.mark.gpu

K_TILES = 16  # sampled whole tiles per frame


def _gpu(sc, tile, ppt, mode, dout=None):
    r = gftorf.Renderer(sc.n, sc.frames, sc.width, sc.height, len(sc.sensor.freqs_hz),
                        len(sc.sensor.offsets_rad), tile=tile, render_mode=mode,
                        pixels_per_thread=ppt)
    p = gftorf.params_from_scene(sc)
    fr, se, co = (gftorf.frames_from_scene(sc), gftorf.sensor_from_scene(sc),
                  gftorf.consts_from_scene(sc))
    bg = torch.as_tensor(sc.bg, device="cuda")
    r.fit_capacity(p, fr, se, co, bg)
    r.preprocess(p, fr, se, co)
    out = r.render_fwd(bg)
    g = None
    if dout is not None:
        g = r.render_bwd(p, bg, torch.as_tensor(dout, device="cuda"))
        g = {k: v.double().cpu().numpy() for k, v in g.items()}
    code, cnt = r.read_status()
    assert code == gftorf.OK
    return out.double().cpu().numpy(), g, cnt


FULL = [  # (workload, expected (n, frames, width, height), tile, ppt, mode, gradients)
    ("batch_300k", (300_000, 16, 640, 480), (16, 16), 4, 0, True),
    ("batch_300k", (300_000, 16, 640, 480), (8, 8), 2, 1, False),
    ("batch_300k", (300_000, 16, 640, 480), (16, 32), 4, 0, False),
    ("batch_300k", (300_000, 16, 640, 480), (16, 32), 4, 1, True),
    ("batch_300k", (300_000, 16, 640, 480), (32, 32), 4, 0, True),
    ("batch_300k", (300_000, 16, 640, 480), (64, 32), 4, 0, True),
    ("batch_300k", (300_000, 16, 640, 480), (64, 64), 4, 1, True),
    ("twofreq_500k", (500_000, 8, 640, 576), (64, 32), 4, 1, False),
    ("dynamic_100k", (100_000, 1, 640, 480), (16, 32), 4, 1, True),
    ("twofreq_500k", (500_000, 8, 640, 576), (16, 32), 4, 1, True),
]


@pytest.mark.parametrize("name,size,tile,ppt,mode,full_grad", FULL)
def test_full_size_sampled_tiles(name, size, tile, ppt, mode, full_grad):
    sc = scenes.make_scene(name, 0, tile=tile)
    assert (sc.n, sc.frames, sc.width, sc.height) == size
    C = sc.n_channels
    tiles = scenes.sample_tiles(sc, K_TILES, seed=9)
    dout = np.zeros((sc.frames, C, sc.height, sc.width), np.float32)
    rng = np.random.default_rng(10)
    refs = []
    for b in range(sc.frames):
        r = ora.render_tiles(sc, b, tiles[b], splats=ora.project(sc, b, ora.EPS_F32))
        refs.append(r)
        keep = r["ambig"] == 0
        px = r["pix"][keep]
        dout[b, :, px[:, 1], px[:, 0]] = rng.standard_normal((keep.sum(), C))
    out, g, cnt = _gpu(sc, tile, ppt, mode, dout if full_grad else None)
    assert cnt > 2 * sc.n * sc.frames  # millions of (Gaussian, tile) instances per frame
    npix = nflag = capped = 0
    worst, worst_alt, kinds = 0.0, 0.0, {}
    for b in range(sc.frames):
        r = refs[b]
        q, pix, amb = r["out"], r["pix"], r["ambig"]
        got = out[b][:, pix[:, 1], pix[:, 0]].T  # (npix, C)
        sigma = np.sqrt((q ** 2).mean(axis=0)) + 1e-30
        flag = (amb & ora.AMB_VALUE) != 0
        npix += len(q)
        nflag += int(flag.sum())
        capped += r["capped"]
        for kind, bit in ora.AMB.items():
            kinds[kind] = kinds.get(kind, 0) + int(((amb & bit) != 0).sum())
        err = np.abs(got - q) / np.maximum(np.abs(q), sigma[None, :])
        worst = max(worst, float(err[~flag].max()))
        for i in np.flatnonzero(flag):
            worst_alt = max(worst_alt, match_alternatives(got[i], r["alts"][int(i)], sigma))
    # every pixel of the sampled tiles that lies in the image (64-high tiles
    # overhang 480-row images)
    inside = sum(min(tile[0], sc.width - tx * tile[0]) * min(tile[1], sc.height - ty * tile[1])
                 for b in range(sc.frames) for tx, ty in tiles[b])
    assert npix == inside
    # every sampled pixel equals a valid oracle result: the nominal walk, or
    # (near-threshold decisions) the walk that decided them the same way
    assert worst <= 1e-5, worst
    assert worst_alt <= 1e-5, (worst_alt, nflag, kinds)
    assert capped == 0, capped
    if full_grad:
        g_ora = ora.backward(sc, dout.astype(np.float64))
        for k, (nrm, elem) in grads_close(g, g_ora, absent=absent_groups(sc)).items():
            assert nrm <= 1e-3 and elem <= 1e-3, (k, nrm, elem)


def test_mlp_full_size_sampled_rows():
    """The deformation MLP at the benchmark's size (300k Gaussians x 16
    timesteps = 4.8M rows) in the fused kernels bench.py times: offsets of
    sampled rows against the BF16 oracle, the inference kernel bit-identical to
    the training forward, and the gradients of a loss that only sees the
    sampled rows (dL/d(delta) zero elsewhere), which the oracle computes
    exactly from those rows alone.  Bars: the whole-network ones (output
    2e-3, gradients 2.5e-2 per layer, norm-wise)."""
    from oracle import mlp as omlp
    from paper_2505_05356_gb300 import mlp

    N, B, K = 300_000, 16, 384
    theta = scenes.init_mlp_params(0, head_std=0.05)
    rng = np.random.default_rng(21)
    means = rng.uniform(-2.0, 4.0, (N, 3)).astype(np.float32)
    times = list(np.linspace(0.0, 1.0, B).astype(np.float32))
    inv = np.float32(1.0 / mlp.unambiguous_range(30e6))
    rows = np.sort(rng.choice(N * B, K, replace=False))
    dd = np.zeros((B * N, 3), np.float32)
    dd[rows] = rng.standard_normal((K, 3)).astype(np.float32)

    net = mlp.DeformationMLP(N, B, float(inv))
    th = torch.as_tensor(theta, device="cuda")
    mu = torch.as_tensor(means, device="cuda")
    delta = net.forward(th, mu, times).clone()
    d_theta, d_means = net.backward(th, mu, times, torch.as_tensor(dd.reshape(B, N, 3),
                                                                   device="cuda"))
    infer = net.infer(th, mu, times)
    torch.cuda.synchronize()
    net.check()
    np.testing.assert_array_equal(infer.cpu().numpy(), delta.cpu().numpy())

    # the oracle on the sampled rows only
    b_of, g_of = rows // N, rows % N
    enc = np.concatenate([omlp.encode(means[g:g + 1], np.asarray([times[b]], np.float64), inv,
                                      single=True) for b, g in zip(b_of, g_of)])
    d_o, acts = omlp.forward(theta.astype(np.float64), enc, bf16=True)
    got = delta.double().cpu().numpy().reshape(-1, 3)[rows]
    assert np.linalg.norm(got - d_o) / np.linalg.norm(d_o) < 2e-3
    g_o, denc = omlp.backward(theta.astype(np.float64), acts, dd[rows].astype(np.float64),
                              bf16=True)
    for l, ((W, b), (Wo, bo)) in enumerate(zip(omlp.unpack(d_theta.double().cpu().numpy()),
                                              omlp.unpack(g_o))):
        assert np.linalg.norm(W - Wo) / np.linalg.norm(Wo) < 2.5e-2, l
        assert np.linalg.norm(b - bo) / np.linalg.norm(bo) < 2.5e-2, l
    # dL/d(means) of the sampled rows' Gaussians (all other rows contribute 0)
    dm_o = np.zeros((N, 3))
    for i, (b, g) in enumerate(zip(b_of, g_of)):
        dm_o[g] += omlp.encode_backward(denc[i:i + 1], means[g:g + 1], [times[b]], inv,
                                        single=True)[0]
    gs = np.unique(g_of)
    dm = d_means.double().cpu().numpy()
    assert np.linalg.norm(dm[gs] - dm_o[gs]) / np.linalg.norm(dm_o[gs]) < 2.5e-2
    others = np.setdiff1d(np.arange(N), gs)
    assert np.all(dm[others] == 0.0)
