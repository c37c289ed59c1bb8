"""The binning entry point that allocates nothing.

Some callers cannot allocate device memory (code inside a graph-capture
region, host callbacks, plugins limited to the buffers they are handed), so
the library offers gftorf_sort_footprints_noalloc, which keeps its scratch in
a fixed device array instead of a caller-allocated workspace.  It must give
exactly the lists of the workspace version (integer work: bit-exact), also on
back-to-back calls that reuse the shared array, and refuse problems that do
not fit the array.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from paper_2505_05356_gb300 import gftorf

pytestmark = pytest.mark.gpu


def _footprints(seed, B, n, W, H):
    rng = np.random.default_rng(seed)
    u = rng.uniform(-30, W + 30, (B, n)).astype(np.float32)
    v = rng.uniform(-30, H + 30, (B, n)).astype(np.float32)
    r = rng.integers(-1, 40, (B, n)).astype(np.int32)
    z = rng.uniform(0.2, 6.0, (B, n)).astype(np.float32)
    z[:, 1::7] = z[:, 0:1]  # exact depth ties
    return [torch.as_tensor(a, device="cuda") for a in (u, v, r, z)]


def test_noalloc_matches_workspace_version_on_consecutive_calls():
    W, H, tile = 200, 150, (16, 16)
    for seed, (B, n) in ((3, (2, 5000)), (4, (3, 7000))):  # two calls in a row
        u, v, r, z = _footprints(seed, B, n, W, H)
        keys_ref, vals_ref, ranges_ref = gftorf.sort_footprints(u, v, r, z, W, H, tile)
        m = keys_ref.numel()
        code, keys, vals, ranges, count = gftorf.sort_footprints_noalloc(
            u, v, r, z, W, H, tile, max_instances=m + 100)
        torch.cuda.synchronize()
        assert code == gftorf.OK, gftorf.STATUS.get(code)
        assert int(count.item()) == m
        assert torch.equal(keys[:m], keys_ref)
        assert torch.equal(vals[:m], vals_ref)
        assert torch.equal(ranges, ranges_ref)


def test_noalloc_rejects_problems_larger_than_its_scratch():
    n = 2_000_000  # ~64 MB of per-Gaussian scratch: more than the fixed array
    u = torch.zeros((1, n), device="cuda")
    r = torch.ones((1, n), dtype=torch.int32, device="cuda")
    code, *_ = gftorf.sort_footprints_noalloc(u, u, r, u + 1, 64, 64, (16, 16), max_instances=16)
    assert code == gftorf.ERR_WORKSPACE


def test_noalloc_overflow_leaves_empty_lists_after_a_call_that_fit():
    """Capacity overflow is reported through *count (> max_instances) and
    leaves every range empty, even though the shared array still holds the
    previous call's lists and counters."""
    W, H, tile = 160, 120, (16, 16)
    u, v, r, z = _footprints(5, 2, 4000, W, H)
    keys_ref, _, _ = gftorf.sort_footprints(u, v, r, z, W, H, tile)
    m = keys_ref.numel()
    code, *_ = gftorf.sort_footprints_noalloc(u, v, r, z, W, H, tile, max_instances=m + 10)
    assert code == gftorf.OK
    code, keys, vals, ranges, count = gftorf.sort_footprints_noalloc(
        u, v, r, z, W, H, tile, max_instances=m // 3)
    torch.cuda.synchronize()
    assert code == gftorf.OK, gftorf.STATUS.get(code)
    assert int(count.item()) == m > m // 3
    assert int(ranges.view(torch.int32).abs().sum().item()) == 0
