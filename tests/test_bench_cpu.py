"""bench.py's CPU-side pieces on a small scene (no GPU): the oracle timing
sample (whole tiles, so that per-tile and per-pixel work extrapolate alike)
and the CPU-baseline object of the JSON line."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import oracle as ora  # noqa: E402
from paper_2505_05356_gb300 import scenes  # noqa: E402


def test_oracle_sample_takes_whole_tiles():
    sc = scenes.make_scene("static_1k", 2, n=300, width=72, height=40)
    fps, spent, det = bench.oracle_sample(sc, 600, seed=3)
    TW, TH = sc.consts.tile_w, sc.consts.tile_h
    tiles_x, tiles_y = -(-72 // TW), -(-40 // TH)
    assert 1 <= det["tiles"] <= tiles_x * tiles_y
    # every sampled tile contributes all its pixels inside the image
    assert det["tiles"] * TW * TH >= det["pixels"] >= det["tiles"] * TW * (40 % TH or TH) // TH
    assert fps > 0 and spent > 0
    # the whole frame as the sample: nothing is extrapolated
    fps_all, _, det_all = bench.oracle_sample(sc, 72 * 40, seed=3)
    assert det_all["pixels"] == 72 * 40 and det_all["tiles"] == tiles_x * tiles_y


def test_cpu_baseline_reports_threads_and_single_thread_rate():
    sc = scenes.make_scene("static_1k", 2, n=300, width=72, height=40)
    threads = ora.num_threads()
    cb = bench.cpu_baseline(sc, 0.5)
    assert ora.num_threads() == threads  # restored after the one-thread sample
    assert cb["kind"] == "oracle" and cb["cores"] == threads and cb["nproc"] == os.cpu_count()
    assert cb["value"] > 0 and cb["single_thread"]["value"] > 0
    assert "tile" in cb["sample"] and cb["unit"] == bench.UNIT
    assert np.isfinite(cb["value"])
