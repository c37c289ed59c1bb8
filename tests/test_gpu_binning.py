"""Bit-exact binning: the device depth sort + stable tile counting sort equals
the oracle's (key, index) ordering of the 64-bit frame|tile|depth keys on the
same single-precision footprints (integer work: no tolerance)."""
import numpy as np
import pytest
import torch

from oracle import oracle as ora
from paper_2505_05356_gb300 import gftorf

pytestmark = pytest.mark.gpu


def _footprints(seed, B, n, W, H, rmax=30, tie_frac=0.05):
    rng = np.random.default_rng(seed)
    u = rng.uniform(-40, W + 40, (B, n)).astype(np.float32)
    v = rng.uniform(-40, H + 40, (B, n)).astype(np.float32)
    r = rng.integers(-2, rmax, (B, n)).astype(np.int32)
    z = rng.uniform(0.2, 8.0, (B, n)).astype(np.float32)
    # exact depth ties (broken by index) and duplicated footprints
    k = int(tie_frac * n)
    if k:
        idx = rng.choice(n, (B, k))
        for b in range(B):
            z[b, idx[b]] = z[b, 0]
    # tile-boundary centres: u - r lands exactly on multiples of 8
    k2 = max(1, n // 50)
    for b in range(B):
        j = rng.choice(n, k2, replace=False)
        u[b, j] = (rng.integers(0, W // 8 + 1, k2) * 8 + r[b, j]).astype(np.float32)
    return u, v, r, z


def _compare(u, v, r, z, W, H, tile):
    keys_o, vals_o, ranges_o = ora.bin_f32(u, v, r, z, W, H, *tile)
    dev = "cuda"
    keys, vals, ranges = gftorf.sort_footprints(*(torch.as_tensor(a).to(dev) for a in (u, v, r, z)),
                                                W, H, tile)
    keys = keys.cpu().numpy().view(np.uint64)
    vals = vals.cpu().numpy().view(np.uint32)
    ranges = ranges.cpu().numpy().view(np.uint32)
    assert keys.shape == keys_o.shape
    np.testing.assert_array_equal(keys, keys_o)
    np.testing.assert_array_equal(vals, vals_o)
    np.testing.assert_array_equal(ranges, ranges_o)
    return len(keys)


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (16, 32)])
@pytest.mark.parametrize("shape", [(1, 500, 64, 64), (3, 2000, 100, 70), (2, 9000, 200, 150)])
def test_sort_matches_oracle_bit_exact(tile, shape):
    B, n, W, H = shape
    u, v, r, z = _footprints(sum(shape) + tile[0], B, n, W, H)
    m = _compare(u, v, r, z, W, H, tile)
    assert m > n  # several tiles per Gaussian on average


def test_sort_edge_cases():
    W, H = 37, 29  # ragged: partial tiles on both edges
    # all invisible
    u, v, r, z = _footprints(1, 2, 300, W, H)
    r[:] = 0
    assert _compare(u, v, r, z, W, H, (16, 16)) == 0
    # one Gaussian covering everything; non-finite centres are never visible
    u, v, r, z = _footprints(2, 1, 64, W, H)
    r[0, 0] = 10000
    u[0, 5] = np.nan
    v[0, 6] = np.inf
    u[0, 7] = -1e30
    _compare(u, v, r, z, W, H, (8, 8))
    # all depths equal: order is by index inside each tile
    u, v, r, z = _footprints(3, 2, 700, W, H)
    z[:] = 1.5
    _compare(u, v, r, z, W, H, (16, 16))


def test_sort_many_chunks_and_sort_tiles():
    """More Gaussians than one depth-sort tile (4096) and one binning chunk."""
    B, n, W, H = 2, 30000, 320, 240
    u, v, r, z = _footprints(9, B, n, W, H, rmax=20, tie_frac=0.01)
    _compare(u, v, r, z, W, H, (16, 16))


def _oracle_footprints(sc):
    """The oracle's single-precision footprints of every frame of `sc`: (u, v,
    3-sigma radius (0: culled), view depth), each (B, N)."""
    S = ora.SP
    u, v, r, z = [], [], [], []
    for b in range(sc.frames):
        sp = ora.project(sc, b)
        vis = sp[:, S["VIS"]] != 0
        u.append(sp[:, S["U"]].astype(np.float32))
        v.append(sp[:, S["V"]].astype(np.float32))
        r.append(np.where(vis, sp[:, S["RAD"]], 0).astype(np.int32))
        z.append(sp[:, S["Z"]].astype(np.float32))
    return [np.ascontiguousarray(np.stack(a)) for a in (u, v, r, z)]


@pytest.mark.parametrize("tile,least", [((16, 32), 40_000_000), ((32, 32), 25_000_000),
                                        ((64, 32), 14_000_000)])
def test_sort_matches_oracle_bit_exact_at_benchmark_density(tile, least):
    """The benchmark's density: 300k Gaussians x 16 frames at 640x480 with
    16x32, 32x32 and 64x32 tiles (tens of millions of instances, thousands of
    binning chunks, full-width scans), footprints as the oracle projects
    them, sorted by gftorf_sort_footprints and by the oracle's (key, index)
    sort."""
    from paper_2505_05356_gb300 import scenes
    sc = scenes.make_scene("batch_300k", 0, tile=tile)
    u, v, r, z = _oracle_footprints(sc)
    m = _compare(u, v, r, z, sc.width, sc.height, tile)
    assert m > least


def test_pipeline_lists_match_oracle_rects_full_size():
    """The pipeline's own lists (preprocess + binning, culling off) for the
    full-size 100k-Gaussian frame against the oracle's FP64 3-sigma tile
    rectangles: the same (tile, Gaussian) pairs except boundary flips (a tile
    inside the oracle's outer rectangle but not its inner one), in depth
    order within each tile."""
    from paper_2505_05356_gb300 import scenes
    from tests.gpu_helpers import run_gpu
    sc = scenes.make_scene("dynamic_100k", 6)
    res = run_gpu(sc, flags=gftorf.FLAG_NO_TILE_CULL)
    _, vals, ranges, count = res["renderer"].tile_lists(with_keys=False)
    m = int(count.item())
    vals = vals[:m].cpu().numpy().astype(np.int64)
    ranges = ranges.cpu().numpy().astype(np.int64)
    T, tx_n = res["renderer"].n_tiles, res["renderer"].tiles_x
    tile_of = np.repeat(np.arange(T), ranges[:, 1] - ranges[:, 0])
    gpu_pairs = tile_of * sc.n + vals
    S = ora.SP
    sp = ora.project(sc, 0, ora.EPS_F32)
    vis = np.flatnonzero(sp[:, S["VIS"]] != 0)

    def pairs_of(prefix, gs):
        x0, y0 = sp[gs, S[prefix + "X0"]].astype(np.int64), sp[gs, S[prefix + "Y0"]].astype(np.int64)
        x1, y1 = sp[gs, S[prefix + "X1"]].astype(np.int64), sp[gs, S[prefix + "Y1"]].astype(np.int64)
        w, h = np.maximum(x1 - x0, 0), np.maximum(y1 - y0, 0)
        n = w * h
        g = np.repeat(gs, n)
        k = np.arange(n.sum()) - np.repeat(np.cumsum(n) - n, n)
        tx = np.repeat(x0, n) + k % np.repeat(np.maximum(w, 1), n)
        ty = np.repeat(y0, n) + k // np.repeat(np.maximum(w, 1), n)
        return np.unique((ty * tx_n + tx) * sc.n + g)

    ora_pairs = pairs_of("", vis)
    only_gpu = np.setdiff1d(gpu_pairs, ora_pairs)
    only_ora = np.setdiff1d(ora_pairs, gpu_pairs)
    may = pairs_of("M", np.arange(sc.n))
    sure = pairs_of("I", vis)
    # every difference is a boundary flip
    assert np.all(np.isin(only_gpu, may)) and not np.any(np.isin(only_gpu, sure))
    assert not np.any(np.isin(only_ora, sure))
    flips = len(only_gpu) + len(only_ora)
    assert len(ora_pairs) > 2_000_000
    assert flips <= 1e-5 * len(ora_pairs), flips
    # depth order within each tile (the oracle's view depth)
    zz = sp[vals, S["Z"]]
    same_tile = tile_of[1:] == tile_of[:-1]
    assert np.all((np.diff(zz) >= -1e-6 * np.abs(zz[1:]))[same_tile])
