"""The seeded synthetic workloads follow their stated recipe (shapes,
distributions, per-frame visibility, sensor), and the autotuner offers only
launch configurations the library accepts.  CPU only."""
import math

import numpy as np
import pytest

from paper_2505_05356_gb300 import autotune, scenes


def test_batch_workload_recipe():
    sc = scenes.make_scene("batch_300k", 0)
    assert (sc.n, sc.frames, sc.width, sc.height) == (300_000, 16, 640, 480)
    # timesteps uniform in [0, 1]
    np.testing.assert_allclose(sc.times, np.arange(16) / 15, atol=1e-7)
    # depths in [1, 3] m, laterally inside the frustum at that depth
    z = sc.means[:, 2]
    assert z.min() >= 1.0 and z.max() <= 3.0
    cam = sc.cameras[0]
    assert np.all(np.abs(sc.means[:, 0]) <= (cam.width / 2) / cam.fx * z * (1 + 1e-6))
    assert np.all(np.abs(sc.means[:, 1]) <= (cam.height / 2) / cam.fy * z * (1 + 1e-6))
    # log-scales N(-3.5, 0.3), unit quaternions, sigmoid(N(0,1)) opacity, U(0.1, 1) amplitude
    ls = np.log(sc.scales.astype(np.float64))
    assert abs(ls.mean() + 3.5) < 0.01 and abs(ls.std() - 0.3) < 0.01
    np.testing.assert_allclose(np.linalg.norm(sc.quats, axis=1), 1.0, atol=1e-6)
    assert 0.0 < sc.opacity.min() and sc.opacity.max() < 1.0
    assert abs(np.median(sc.opacity) - 0.5) < 0.01
    assert sc.amplitude.min() >= 0.1 and sc.amplitude.max() <= 1.0
    # cubic trajectory coefficients N(0, 0.05) m
    assert abs(sc.coeffs.std() - 0.05) < 0.002
    # 30-100 % of the Gaussians visible per frame: the rest shifted out of
    # the frustum by 10 m for that frame only
    shifted = sc.delta[:, :, 0] == 10.0
    assert np.all((sc.delta[:, :, 0] == 0.0) | shifted)
    assert np.all(sc.delta[:, :, 1:] == 0.0)
    vis = 1.0 - shifted.mean(axis=1)
    assert vis.min() >= 0.3 - 0.01 and vis.max() <= 1.0 and vis.std() > 0.05
    # 30 MHz, four offsets, raw quartet + ambient, background U(-1, 1)
    assert sc.sensor.freqs_hz == [30e6] and len(sc.sensor.offsets_rad) == 4
    assert sc.n_channels == 5 and sc.bg.shape == (16, 5)
    assert np.all(np.abs(sc.bg) <= 1.0)


def test_other_workload_recipes():
    one = scenes.make_scene("static_1k", 0)
    assert (one.n, one.frames, one.width, one.height) == (1000, 1, 64, 64)
    assert np.all(np.abs(one.means[:, :2]) <= 0.5) and one.means[:, 2].min() >= 1.0
    assert one.coeffs is None and one.delta is None
    two = scenes.make_scene("twofreq_500k", 0, n=20_000)
    assert (two.frames, two.width, two.height) == (8, 640, 576)
    assert two.sensor.freqs_hz == [30e6, 80e6] and two.n_channels == 9
    assert two.means[:, 2].min() >= 0.5 and two.means[:, 2].max() <= 6.0
    dyn = scenes.make_scene("dynamic_100k", 0, n=5000)
    assert dyn.frames == 1 and 0.0 <= float(dyn.times[0]) <= 1.0 and dyn.delta is None


def test_async_capture_recipe():
    sc = scenes.make_scene("batch_300k", 3, n=2000, frames=8, async_capture=True)
    assert len(sc.sensor.offsets_rad) == 1 and sc.n_channels == 2
    np.testing.assert_allclose(sc.frame_phase, [(math.pi / 2) * (b % 4) for b in range(8)],
                               atol=1e-6)
    tick = 1.0 / 7
    for b in range(8):
        t0, t1 = sc.interp_times[b]
        assert t0 == pytest.approx(4 * (b // 4) * tick, abs=1e-6)
        assert t1 == pytest.approx(t0 + 4 * tick, abs=1e-6)


def test_seeded_workloads_are_reproducible():
    a = scenes.make_scene("batch_300k", 5, n=3000, frames=3)
    b = scenes.make_scene("batch_300k", 5, n=3000, frames=3)
    c = scenes.make_scene("batch_300k", 6, n=3000, frames=3)
    np.testing.assert_array_equal(a.means, b.means)
    np.testing.assert_array_equal(a.delta, b.delta)
    assert not np.array_equal(a.means, c.means)


def test_autotune_candidates_are_accepted_launch_shapes():
    cands = autotune.candidates()
    assert len(cands) == len({(tuple(c["tile"]), c["ppt"], c["mode"]) for c in cands})
    for c in cands:
        tw, th = c["tile"]
        assert (tw, th) in autotune.TILES and c["mode"] in (0, 1)
        assert tw * th // c["ppt"] >= 32  # a full warp per tile
        assert th % c["ppt"] == 0          # whole columns of pixels per thread
    # the 8x8 tile with 4 pixels per thread (16 threads) is not offered, and
    # 32-wide tiles only with 4 pixels per thread
    assert not any(tuple(c["tile"]) == (8, 8) and c["ppt"] == 4 for c in cands)
    assert not any(c["tile"][0] == 32 and c["ppt"] != 4 for c in cands)
    assert any(tuple(c["tile"]) == (32, 32) for c in cands)
