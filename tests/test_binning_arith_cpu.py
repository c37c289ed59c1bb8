"""Integer arithmetic the binning kernels take on trust, checked on the CPU.

The ordered scatter splits an instance's row-major index `local` inside its
Gaussian's tile rectangle (width w) into (row, column) from an approximate
single-precision reciprocal of w and one exact correction step.  That is
right whenever the truncated quotient is off by at most one, which holds if
the reciprocal's relative error stays well below 1 / local.  The kernels'
reciprocal (rcp.approx) is accurate to about 2^-23; here every index below
50000 (the most tiles a frame may have) and every width up to 2048 is split
with reciprocals perturbed by a relative 2^-20 either way, and the corrected
split must be exact."""
import numpy as np


def _split(local, inv, w):
    ky = np.trunc(local.astype(np.float32) * inv).astype(np.int64)
    kx = local - ky * w
    lo = kx < 0
    ky[lo] -= 1
    kx[lo] += w
    hi = kx >= w
    ky[hi] += 1
    kx[hi] -= w
    return ky, kx


def test_rectangle_index_split_with_an_approximate_reciprocal():
    local = np.arange(50_000, dtype=np.int64)
    for w in range(1, 2049):
        exact = np.float32(1.0) / np.float32(w)
        for rel in (-2.0 ** -20, 0.0, 2.0 ** -20):
            inv = np.float32(exact * (1.0 + rel))
            ky, kx = _split(local, inv, w)
            np.testing.assert_array_equal(ky, local // w)
            np.testing.assert_array_equal(kx, local % w)
