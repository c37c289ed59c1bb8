"""GPU parity of the CUDA path against the FP64 oracle (through the C ABI).

Bars: tile lists and sort order bit-exact; forward raw samples within 1e-5 of
max(|Q|, channel RMS); gradients within 1e-3 (norm-wise per parameter group
and elementwise against max(|g|, group RMS)).  Pixels where single precision
may take one of the method's discrete decisions (alpha floor, early stop,
depth order, tile membership) the other way have several valid results: each
must equal, at the same 1e-5 bar, one of the oracle's walks with those
decisions taken either way.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as ora
from paper_2505_05356_gb300 import gftorf, scenes
from tests.gpu_helpers import (absent_groups, ambiguous_pixels_match, forward_close,
                               grads_close, run_gpu)

pytestmark = pytest.mark.gpu

POSE = ((4.0, -6.0, 3.0), (0.1, -0.05, -0.2))

SMALL = [
    ("static_1k", dict()),
    ("static_1k", dict(width=50, height=37)),
    ("static_1k", dict(tile=(8, 8), width=72, height=40)),
    ("static_1k", dict(tile=(16, 32), width=70, height=75)),
    ("static_1k", dict(tile=(32, 32), width=70, height=75)),
    ("static_1k", dict(tile=(64, 32), width=70, height=75)),
    ("static_1k", dict(tile=(64, 64), width=70, height=75)),
    ("static_1k", dict(freqs_hz=[30e6, 80e6], z_range=(0.5, 6.0))),
    ("static_1k", dict(offsets_rad=[0.1, 0.9, 2.0, 2.5, 3.3, 4.0, 5.1, 6.0])),
    ("dynamic_100k", dict(n=3000, width=96, height=80, frames=3)),
    ("batch_300k", dict(n=4000, width=80, height=64, frames=4)),
    ("batch_300k", dict(n=3000, width=72, height=56, frames=2, phasor=True, depth=True)),
    ("static_1k", dict(freqs_hz=[30e6, 80e6], z_range=(0.5, 6.0), phasor=True, depth=True,
                       tile=(16, 32))),
    ("static_1k", dict(sh_degree=0)),
    ("static_1k", dict(sh_degree=1)),
    ("batch_300k", dict(n=3000, width=72, height=56, frames=3, sh_degree=3, sh_std=0.1)),
    ("batch_300k", dict(n=2000, width=64, height=48, frames=2, sh_degree=2, depth=True)),
    # a moved camera (rotation + translation): the SH direction is a world-space
    # direction, no longer the camera-frame one
    ("batch_300k", dict(n=3000, width=72, height=56, frames=3, pose=POSE)),
    ("batch_300k", dict(n=3000, width=72, height=56, frames=3, sh_degree=3, sh_std=0.1,
                        pose=POSE)),
    ("static_1k", dict(sh_degree=1, pose=((3.0, -5.0, 8.0), (0.05, -0.1, -0.3)))),
    # asynchronous raw capture: one offset per frame, Eq. 7 motion between quartets
    ("batch_300k", dict(n=3000, width=72, height=56, frames=8, async_capture=True)),
    ("dynamic_100k", dict(n=3000, width=64, height=48, frames=5, async_capture=True,
                          freqs_hz=[30e6, 80e6], z_range=(0.5, 6.0))),
]

def _ids(case):
    name, kw = case
    return name + "-" + "-".join("%s=%s" % (k, v) for k, v in sorted(kw.items()))


@pytest.mark.parametrize("case", SMALL, ids=[_ids(c) for c in SMALL])
def test_forward_matches_oracle(case):
    name, kw = case
    sc = scenes.make_scene(name, 11, **kw)
    q_ora, tf_ora, amb, nc = ora.render(sc, ora.EPS_F32)
    res = run_gpu(sc)
    assert res["status"][0] == gftorf.OK
    ok, worst, nflag = forward_close(res["out"], q_ora, amb, rel=1e-5)
    assert ok, worst
    keep = (amb & ora.AMB_VALUE) == 0
    np.testing.assert_allclose(res["tfinal"][keep], tf_ora[keep], rtol=2e-5, atol=1e-9)
    # ambiguous pixels: each equals one of the oracle's valid results
    for b in range(sc.frames):
        n_b, worst_b, capped = ambiguous_pixels_match(sc, b, res["out"][b], q_ora[b], amb[b])
        assert capped == 0
        assert worst_b <= 1e-5, (b, n_b, worst_b)


@pytest.mark.parametrize("case", SMALL, ids=[_ids(c) for c in SMALL])
def test_backward_matches_oracle(case):
    name, kw = case
    sc = scenes.make_scene(name, 12, **kw)
    q_ora, tf_ora, amb, nc = ora.render(sc, ora.EPS_F32)
    dout = scenes.random_dout(sc, 3)
    dout[np.broadcast_to((amb != 0)[:, None], dout.shape)] = 0.0  # ambiguous pixels
    g_ora = ora.backward(sc, dout.astype(np.float64))
    res = run_gpu(sc, dout)
    errs = grads_close(res["grads"], g_ora, absent=absent_groups(sc))
    for k, (nrm, elem) in errs.items():
        assert nrm <= 1e-3 and elem <= 1e-3, (k, nrm, elem)
    assert "means" in errs and "opacity" in errs and "bg" in errs
    if kw.get("sh_degree") is not None:
        assert "sh" in errs


FP64_CASES = [dict(freqs_hz=[30e6, 80e6], phasor=True, depth=True),
              dict(sh_degree=3, sh_std=0.1, pose=((4.0, -6.0, 3.0), (0.1, -0.05, -0.2))),
              dict(async_capture=True)]


@pytest.mark.parametrize("kw", FP64_CASES, ids=["phasor-depth", "sh3-moved-camera", "async-eq7"])
def test_fp64_path_matches_oracle_tightly(kw):
    """The double-precision instantiation of every kernel agrees with the
    oracle to ~1e-9 (the formulas, not just the tolerance, agree)."""
    sc = scenes.make_scene("batch_300k", 5, n=1500, width=64, height=48, frames=2, **kw)
    eps64 = (1e-9, 1e-10, 1.2e-7, 1e-9)  # depth keys are single precision
    q_ora, tf_ora, amb, nc = ora.render(sc, eps64)
    dout = scenes.random_dout(sc, 4)
    dout[np.broadcast_to((amb != 0)[:, None], dout.shape)] = 0.0
    res = run_gpu(sc, dout, dtype=torch.float64)
    ok, worst, nflag = forward_close(res["out"], q_ora, amb, rel=1e-9)
    assert ok, worst
    g_ora = ora.backward(sc, dout.astype(np.float64))
    for k, (nrm, elem) in grads_close(res["grads"], g_ora, absent=absent_groups(sc)).items():
        assert nrm <= 1e-8 and elem <= 1e-7, (k, nrm, elem)


def test_empty_scene_and_all_culled():
    """All Gaussians behind the camera: Q = bg, T_N = 1, zero gradients."""
    sc = scenes.make_scene("static_1k", 1, n=300, width=40, height=24)
    sc.means = sc.means.copy()
    sc.means[:, 2] = -1.0
    res = run_gpu(sc, scenes.random_dout(sc, 2))
    assert res["status"] == (gftorf.OK, 0)
    for c in range(sc.n_channels):
        assert np.all(res["out"][0, c] == sc.bg[0, c].astype(np.float64))
    assert np.all(res["tfinal"] == 1.0) and np.all(res["nlast"] == 0)
    for k in ("means", "scales", "quats", "opacity", "amplitude"):
        assert np.all(res["grads"][k] == 0.0), k


def test_zero_gaussians():
    sc = scenes.make_scene("static_1k", 1, n=0, width=33, height=17)
    res = run_gpu(sc, scenes.random_dout(sc, 2), capacity=1)
    assert res["status"] == (gftorf.OK, 0)
    np.testing.assert_array_equal(res["out"][0, :, 0, 0], sc.bg[0].astype(np.float64))


def test_capacity_overflow_is_reported_not_faulted():
    sc = scenes.make_scene("static_1k", 2)
    res = run_gpu(sc, capacity=64)
    code, cnt = res["status"]
    assert code == gftorf.ERR_CAPACITY and cnt > 64
    assert np.all(np.isfinite(res["out"]))


@pytest.mark.parametrize("ppt,tile", [(1, None), (2, None), (4, None), (4, (64, 32)), (4, (64, 64))])
def test_persistent_mode_bit_identical(ppt, tile):
    """Persistent CTAs pulling (frame, tile) items -- two per 64-wide tile --
    render exactly like one CTA per item."""
    kw = dict(tile=tile) if tile else {}
    sc = scenes.make_scene("batch_300k", 3, n=5000, width=96, height=64, frames=3, **kw)
    a = run_gpu(sc, render_mode=0, pixels_per_thread=ppt)
    b = run_gpu(sc, render_mode=1, pixels_per_thread=ppt)
    np.testing.assert_array_equal(a["out"], b["out"])
    np.testing.assert_array_equal(a["nlast"], b["nlast"])


@pytest.mark.parametrize("tile,freqs", [((16, 16), [30e6]), ((8, 8), [30e6]),
                                        ((16, 32), [30e6]), ((16, 32), [30e6, 80e6])])
def test_pixels_per_thread_bit_identical(tile, freqs):
    """1, 2 or 4 pixels per compositing thread: same forward bit for bit,
    same gradients up to atomic summation order."""
    sc = scenes.make_scene("batch_300k", 8, n=4000, width=72, height=56, frames=2,
                           tile=tile, freqs_hz=freqs)
    dout = scenes.random_dout(sc, 5)
    ref = run_gpu(sc, dout, pixels_per_thread=1)
    for ppt in (2, 4):
        if tile[0] * tile[1] // ppt < 32:
            continue
        res = run_gpu(sc, dout, pixels_per_thread=ppt)
        np.testing.assert_array_equal(res["out"], ref["out"])
        np.testing.assert_array_equal(res["nlast"], ref["nlast"])
        for k, (nrm, elem) in grads_close(res["grads"], ref["grads"]).items():
            assert nrm <= 1e-5, (ppt, k, nrm)


@pytest.mark.parametrize("freqs,extra", [([30e6], False), ([30e6, 80e6], True)])
def test_tile_shapes_render_identically(freqs, extra):
    """Every pixel composites the same Gaussians in the same (depth) order
    whatever the tile shape, so the forward is bit-identical across shapes
    (and the gradients equal up to atomic summation order); this also checks
    the 32x32 tile's thread layout (16x8 warp blocks, two across)."""
    sc = scenes.make_scene("batch_300k", 18, n=5000, width=100, height=70, frames=2,
                           freqs_hz=freqs, phasor=extra, depth=extra)
    dout = scenes.random_dout(sc, 7)
    runs = {}
    for tile, ppt in (((16, 32), 4), ((32, 32), 4), ((64, 32), 4), ((64, 64), 4), ((16, 16), 2),
                      ((8, 8), 1)):
        sc.consts.tile_w, sc.consts.tile_h = tile
        runs[tile] = run_gpu(sc, dout, pixels_per_thread=ppt)
    ref = runs[(16, 32)]
    for tile, res in runs.items():
        assert res["status"][0] == gftorf.OK
        np.testing.assert_array_equal(res["out"], ref["out"], err_msg=str(tile))
        np.testing.assert_array_equal(res["tfinal"], ref["tfinal"], err_msg=str(tile))
        for k, (nrm, elem) in grads_close(res["grads"], ref["grads"]).items():
            assert nrm <= 1e-5, (tile, k, nrm)


def test_batched_equals_per_frame():
    """A batch of frames renders exactly like the frames one at a time."""
    sc = scenes.make_scene("batch_300k", 4, n=5000, width=80, height=48, frames=4)
    full = run_gpu(sc)
    for b in range(sc.frames):
        one = scenes.Scene(sc.means, sc.coeffs, sc.scales, sc.quats, sc.opacity,
                           sc.amplitude, sc.times[b:b + 1], sc.cameras[b:b + 1],
                           sc.delta[b:b + 1], sc.sensor, sc.consts, sc.bg[b:b + 1])
        r = run_gpu(one)
        np.testing.assert_array_equal(full["out"][b], r["out"][0])


@pytest.mark.parametrize("tile,ppt", [((16, 16), 2), ((16, 32), 4), ((8, 8), 1), ((64, 32), 4),
                                      ((64, 64), 4)])
def test_tile_culling_changes_nothing(tile, ppt):
    """Dropping (Gaussian, tile) pairs that cannot reach alpha_min anywhere in
    the tile leaves the forward bit-identical and the gradients equal up to
    atomic summation order, with fewer instances."""
    sc = scenes.make_scene("batch_300k", 9, n=6000, width=96, height=80, frames=3, tile=tile)
    dout = scenes.random_dout(sc, 6)
    on = run_gpu(sc, dout, pixels_per_thread=ppt)
    off = run_gpu(sc, dout, pixels_per_thread=ppt, flags=gftorf.FLAG_NO_TILE_CULL)
    np.testing.assert_array_equal(on["out"], off["out"])
    np.testing.assert_array_equal(on["tfinal"], off["tfinal"])
    for k, (nrm, elem) in grads_close(on["grads"], off["grads"]).items():
        assert nrm <= 1e-5, (k, nrm)
    # fewer instances (a 64-wide tile's box is dropped less often)
    assert on["status"][1] < (1.0 if tile[0] == 64 else 0.95) * off["status"][1]


BINNING_SCENES = [  # (workload, overrides, flips allowed per (Gaussian, tile) pair)
    ("static_1k", dict(), 0.0),                                     # config 1, full size
    ("dynamic_100k", dict(n=3000, width=96, height=80), 0.0),       # config 2's shape
    ("batch_300k", dict(n=3000, width=96, height=80, frames=2), 1e-3),
    ("batch_300k", dict(n=3000, width=130, height=80, frames=2, tile=(64, 32)), 1e-3),
]


@pytest.mark.parametrize("flags", [0, gftorf.FLAG_NO_TILE_CULL])
@pytest.mark.parametrize("name,over,flip_rate", BINNING_SCENES)
def test_tile_lists_match_oracle_binning_of_its_own_rects(flags, name, over, flip_rate):
    """The pipeline's instance lists against the oracle's FP64 3-sigma
    rectangles.  A membership difference is a boundary flip when the tile is
    inside the oracle's outer (may-cover) rectangle but not its inner
    (surely-covers) one: single-precision rounding can put it either side.
    Without culling every difference must be a flip; with culling the lists
    may also drop pairs, each with alpha < alpha_min at every pixel centre of
    the tile.  Flips are counted: none on the two single-frame workloads."""
    sc = scenes.make_scene(name, 6, **over)
    res = run_gpu(sc, flags=flags)
    keys, vals, ranges, count = res["renderer"].tile_lists()
    m = int(count.item())
    vals = vals[:m].cpu().numpy()
    ranges = ranges.cpu().numpy()
    T = res["renderer"].n_tiles
    tx_n = res["renderer"].tiles_x
    amin = sc.consts.alpha_min
    TW, TH = sc.consts.tile_w, sc.consts.tile_h
    SPI = ora.SP
    flips, pairs = 0, 0
    for b in range(sc.frames):
        sp = ora.project(sc, b, ora.EPS_F32)
        vis = sp[:, SPI["VIS"]] != 0

        def inside(tx, ty, k):
            return ((sp[:, SPI[k + "X0"]] <= tx) & (tx < sp[:, SPI[k + "X1"]]) &
                    (sp[:, SPI[k + "Y0"]] <= ty) & (ty < sp[:, SPI[k + "Y1"]]))

        for t in range(T):
            tx, ty = t % tx_n, t // tx_n
            s, e = ranges[b * T + t]
            gpu_set = set(vals[s:e].tolist())
            inr = inside(tx, ty, "") & vis
            sure = inside(tx, ty, "I")
            may = inside(tx, ty, "M")
            ora_set = set(np.nonzero(inr)[0].tolist())
            pairs += len(ora_set)
            for g in gpu_set - ora_set:  # listed by the GPU only: a flip
                assert may[g] and not sure[g], (b, t, g)
                flips += 1
            for g in ora_set - gpu_set:
                if not flags:  # culling on: a pair no pixel of the tile reaches
                    xs = np.arange(tx * TW, (tx + 1) * TW) + 0.5
                    ys = np.arange(ty * TH, (ty + 1) * TH) + 0.5
                    X, Y = np.meshgrid(xs, ys)
                    dx, dy = sp[g, SPI["U"]] - X, sp[g, SPI["V"]] - Y
                    pw = -0.5 * (sp[g, SPI["CA"]] * dx * dx + sp[g, SPI["CC"]] * dy * dy) \
                        - sp[g, SPI["CB"]] * dx * dy
                    if (sp[g, SPI["OPA"]] * np.exp(pw)).max() < amin * (1 + 1e-4):
                        continue
                assert not sure[g], (b, t, g)  # otherwise only a flip the other way
                flips += 1
            # depth order within the tile (view depth of the oracle)
            z = sp[vals[s:e], SPI["Z"]]
            assert np.all(np.diff(z) >= -1e-6 * np.abs(z[1:])), (b, t)
    assert pairs > 1000
    assert flips <= flip_rate * pairs, (flips, pairs)


def test_async_frame_equals_channel_of_synchronous_quartet():
    """One raw frame that samples offset phi_j (P = 1, the frame's own phase
    offset) is bit-identical to channel j of the synchronous quartet."""
    import math
    sync = scenes.make_scene("batch_300k", 14, n=4000, width=80, height=64, frames=1)
    rs = run_gpu(sync)
    offs = sync.sensor.offsets_rad
    for j in range(4):
        one = scenes.make_scene("batch_300k", 14, n=4000, width=80, height=64, frames=1)
        one.sensor.offsets_rad = [0.0]
        one.frame_phase = np.array([offs[j]], np.float32)
        one.bg = np.stack([sync.bg[:, j], sync.bg[:, 4]], 1)
        r1 = run_gpu(one)
        np.testing.assert_array_equal(r1["out"][0, 0], rs["out"][0, j])
        np.testing.assert_array_equal(r1["out"][0, 1], rs["out"][0, 4])
    assert abs(offs[1] - math.pi / 2) < 1e-6


def test_telescoping_coincident_gaussians_on_the_gpu():
    """The golden telescoping case through the CUDA path's own outputs: N
    coincident Gaussians of equal alpha with unit amplitude term A = s r / d^2
    and zero background, so the ambient channel is sum_k alpha T_k^2 (the
    golden geometric series) and the exported T_N is (1 - alpha)^N."""
    import json
    import os
    from tests.oracle_scenes import at_pixel, tiny_scene
    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                         "closed_forms.json")))
    case = golden["telescoping"]["cases"][0]
    cam = tiny_scene([[0, 0, 1]], 0.1).cameras[0]
    p = at_pixel(cam, 10.5, 50.5, 2.0)
    d = float(np.linalg.norm(p))
    n = case["N"]
    sc = tiny_scene([p] * n, 0.05, opacity=[case["alpha"]] * n, amplitude=[d * d] * n)
    res = run_gpu(sc)
    assert res["out"][0, 4, 50, 10] == pytest.approx(case["sum_weights"], rel=1e-5)
    assert res["tfinal"][0, 50, 10] == pytest.approx(case["T_final"], rel=1e-5)
    assert res["nlast"][0, 50, 10] >= n  # all N composited (list position past the last)
