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
