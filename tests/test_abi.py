"""C-ABI library checks that need no GPU: it builds, loads, exports every
symbol include/gftorf.h declares, sizes workspaces and rejects invalid
arguments on the host before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2505_05356_gb300 import gftorf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "gftorf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gftorf_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    return gftorf.load()


def test_exports_every_declared_symbol(lib):
    names = _declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_status_strings(lib):
    assert lib.gftorf_version() == 101
    for code, text in gftorf.STATUS.items():
        assert lib.gftorf_status_string(code).decode() == text


def _dims(**kw):
    d = dict(n_gaussians=1000, n_frames=2, width=64, height=48, tile_w=16, tile_h=16,
             n_freq=1, n_offsets=4, dtype=0, render_mode=0, pixels_per_thread=0,
             flags=0, n_sh=0, reserved=0, max_instances=10000)
    d.update(kw)
    return gftorf.Dims(*[d[k] for k, _ in gftorf.Dims._fields_])


def test_workspace_size_validates_dims(lib):
    ok = lib.gftorf_workspace_size(ctypes.byref(_dims()))
    assert ok > 0 and ok % 256 == 0
    # more capacity, frames or precision never shrink the workspace
    assert lib.gftorf_workspace_size(ctypes.byref(_dims(max_instances=20000))) >= ok + 40000 - 256
    assert lib.gftorf_workspace_size(ctypes.byref(_dims(dtype=1))) > ok
    assert lib.gftorf_workspace_size(ctypes.byref(_dims(n_frames=4))) > ok
    for bad in (dict(n_frames=0), dict(n_frames=65), dict(width=0), dict(tile_w=12),
                dict(tile_w=32, tile_h=16), dict(n_freq=0), dict(n_freq=5),
                dict(n_offsets=9), dict(dtype=2), dict(render_mode=2),
                dict(pixels_per_thread=3), dict(pixels_per_thread=8),
                dict(tile_w=8, tile_h=8, pixels_per_thread=4), dict(flags=16),
                dict(n_gaussians=-1), dict(max_instances=-1), dict(n_sh=2),
                dict(n_sh=25), dict(reserved=1),
                dict(max_instances=1 << 33),
                # tiles 32 or more wide take 4 pixels per thread only; no other
                # 64-wide or taller shapes
                dict(tile_w=64, tile_h=32, pixels_per_thread=2),
                dict(tile_w=64, tile_h=64, pixels_per_thread=1),
                dict(tile_w=64, tile_h=16), dict(tile_w=128, tile_h=64),
                dict(tile_w=32, tile_h=64)):
        assert lib.gftorf_workspace_size(ctypes.byref(_dims(**bad))) == 0, bad
    # every binning tile shape, with its pixels per thread
    for tw, th, ppt in ((8, 8, 1), (16, 16, 2), (16, 32, 4), (32, 32, 4), (64, 32, 4),
                        (64, 64, 4), (64, 64, 0)):
        d = _dims(tile_w=tw, tile_h=th, pixels_per_thread=ppt)
        assert lib.gftorf_workspace_size(ctypes.byref(d)) > 0, (tw, th, ppt)
    assert lib.gftorf_workspace_size(None) == 0
    # the empty scene is a valid problem
    assert lib.gftorf_workspace_size(ctypes.byref(_dims(n_gaussians=0))) > 0
    for nsh in (1, 4, 9, 16):
        assert lib.gftorf_workspace_size(ctypes.byref(_dims(n_sh=nsh))) > 0


def test_host_side_argument_errors(lib):
    d = _dims()
    g = gftorf.Gaussians()
    fr = (gftorf.Frame * 2)(*[gftorf.make_frame(50, 50, 32, 24, [1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0],
                                                0.2, 0.0) for _ in range(2)])
    se = gftorf.make_sensor([30e6], [0, 1.57, 3.14, 4.71])
    co = gftorf.make_consts()
    # null parameter pointers with N > 0
    assert lib.gftorf_preprocess(ctypes.byref(d), ctypes.byref(g), fr, ctypes.byref(se),
                                 ctypes.byref(co), None, 0, None) == gftorf.ERR_ARG
    # invalid dims
    bad = _dims(tile_w=3)
    assert lib.gftorf_render_fwd(ctypes.byref(bad), ctypes.c_void_p(16), ctypes.c_void_p(16),
                                 None, 0, None) == gftorf.ERR_ARG
    # missing / misaligned / short workspace (checked before any device call)
    assert lib.gftorf_render_fwd(ctypes.byref(d), ctypes.c_void_p(16), ctypes.c_void_p(16),
                                 None, 0, None) == gftorf.ERR_WORKSPACE
    need = lib.gftorf_workspace_size(ctypes.byref(d))
    assert lib.gftorf_render_fwd(ctypes.byref(d), ctypes.c_void_p(16), ctypes.c_void_p(16),
                                 ctypes.c_void_p(4096 + 8), need, None) == gftorf.ERR_WORKSPACE
    assert lib.gftorf_render_fwd(ctypes.byref(d), ctypes.c_void_p(16), ctypes.c_void_p(16),
                                 ctypes.c_void_p(4096), need - 1, None) == gftorf.ERR_WORKSPACE
    # non-finite camera values are rejected on the host
    pg = gftorf.Gaussians(*([ctypes.c_void_p(256)] * 7))
    # SH reflectivity needs its coefficient array
    dsh = _dims(n_sh=4)
    assert lib.gftorf_preprocess(ctypes.byref(dsh), ctypes.byref(pg), fr, ctypes.byref(se),
                                 ctypes.byref(co), ctypes.c_void_p(4096),
                                 lib.gftorf_workspace_size(ctypes.byref(dsh)),
                                 None) == gftorf.ERR_ARG
    fr[1].fx = float("nan")
    assert lib.gftorf_preprocess(ctypes.byref(d), ctypes.byref(pg), fr, ctypes.byref(se),
                                 ctypes.byref(co), ctypes.c_void_p(4096), need,
                                 None) == gftorf.ERR_ARG
    fr[1].fx = 50.0
    # Eq. 7 bracket out of order
    fr[0].interp_t0, fr[0].interp_t1 = 0.5, 0.25
    assert lib.gftorf_preprocess(ctypes.byref(d), ctypes.byref(pg), fr, ctypes.byref(se),
                                 ctypes.byref(co), ctypes.c_void_p(4096), need,
                                 None) == gftorf.ERR_ARG
    fr[0].interp_t0, fr[0].interp_t1 = 0.0, 0.0
    co.alpha_max = 1.5
    assert lib.gftorf_preprocess(ctypes.byref(d), ctypes.byref(pg), fr, ctypes.byref(se),
                                 ctypes.byref(co), ctypes.c_void_p(4096), need,
                                 None) == gftorf.ERR_ARG
    # backward needs its gradient struct
    assert lib.gftorf_render_bwd(ctypes.byref(d), ctypes.byref(pg), ctypes.c_void_p(16),
                                 ctypes.c_void_p(16), None, ctypes.c_void_p(4096), need,
                                 None) == gftorf.ERR_ARG


def test_struct_layouts_match_header():
    # sizes fixed by the header's field lists (C layout, no hidden padding)
    assert ctypes.sizeof(gftorf.Dims) == 14 * 4 + 8
    assert ctypes.sizeof(gftorf.Frame) == 21 * 4
    assert ctypes.sizeof(gftorf.Sensor) == (4 + 8 + 1) * 4
    assert ctypes.sizeof(gftorf.Consts) == 6 * 4
    assert ctypes.sizeof(gftorf.AdamGroup) == 4 * 8 + 8 + 3 * 4 + 4  # tail padding to 8
    assert ctypes.sizeof(gftorf.Gaussians) == 8 * ctypes.sizeof(ctypes.c_void_p)
    assert ctypes.sizeof(gftorf.Gradients) == 9 * ctypes.sizeof(ctypes.c_void_p)


def test_training_calls_reject_bad_arguments_on_host(lib):
    st = ctypes.c_void_p(4096)
    assert lib.gftorf_train_begin(None, None, 0, 0, None) == gftorf.ERR_ARG
    assert lib.gftorf_train_begin(ctypes.c_void_p(4100), None, 0, 0, None) == gftorf.ERR_ARG
    assert lib.gftorf_train_begin(st, ctypes.c_void_p(256), 1 << 20, 0, None) == gftorf.ERR_ARG
    d64 = _dims(dtype=1)
    assert lib.gftorf_l2_loss(ctypes.byref(d64), ctypes.c_void_p(256), ctypes.c_void_p(256),
                              ctypes.c_void_p(256), st, None) == gftorf.ERR_ARG
    assert lib.gftorf_l2_loss(ctypes.byref(_dims()), None, ctypes.c_void_p(256),
                              ctypes.c_void_p(256), st, None) == gftorf.ERR_ARG
    groups = (gftorf.AdamGroup * 13)()
    assert lib.gftorf_adam_step(groups, 13, 0.9, 0.999, 1e-15, st, None) == gftorf.ERR_ARG
    groups[0] = gftorf.AdamGroup(256, 256, 256, 256, 10, 0.1, 1.0, 0.0)  # lo > hi
    assert lib.gftorf_adam_step(groups, 1, 0.9, 0.999, 1e-15, st, None) == gftorf.ERR_ARG
    assert lib.gftorf_adam_step(groups, 0, 1.5, 0.999, 1e-15, st, None) == gftorf.ERR_ARG
    # nothing to update: returns before touching the device
    assert lib.gftorf_adam_step(groups, 0, 0.9, 0.999, 1e-15, st, None) == gftorf.OK


def test_shard_training_calls_reject_bad_arguments_on_host(lib):
    """The shard variants of the fitting calls check their arguments before
    any launch (a fake, aligned state pointer is never touched)."""
    st = ctypes.c_void_p(4096)
    for n, off, stride in ((4, -1, 8), (4, 5, 8), (4, 0, 3), (4, 0, 1 << 41), (-1, 0, 8)):
        assert lib.gftorf_train_begin_shard(st, ctypes.c_void_p(8192), n, 1, off, stride,
                                            None) == gftorf.ERR_ARG, (n, off, stride)
    assert lib.gftorf_train_begin_shard(None, None, 0, 1, 0, 0, None) == gftorf.ERR_ARG
    d = _dims()
    buf = ctypes.c_void_p(8192)
    for count in (0.0, -3.0, float("inf"), float("nan")):
        assert lib.gftorf_l2_loss_scaled(ctypes.byref(d), buf, buf, buf, st, count,
                                         None) == gftorf.ERR_ARG, count


def test_mlp_calls_reject_bad_arguments_on_host(lib):
    from paper_2505_05356_gb300 import mlp
    L = mlp._lib()
    assert L.gftorf_mlp_param_count() == 256 * 128 + 256 + 7 * (256 * 256 + 256) + 3 * 256 + 3
    assert L.gftorf_mlp_workspace_size(-1, 1) == 0
    assert L.gftorf_mlp_workspace_size(10, 0) == 0
    assert L.gftorf_mlp_workspace_size(10, 65) == 0
    assert L.gftorf_mlp_workspace_size(1 << 26, 2) == 0       # 2^27 rows
    assert L.gftorf_mlp_workspace_size((1 << 26) - 1, 2) > 0
    small = L.gftorf_mlp_workspace_size(1000, 2)
    assert small > 0 and small % 256 == 0
    assert L.gftorf_mlp_workspace_size(2000, 2) > small
    t = (ctypes.c_float * 2)(0.0, 1.0)
    ws = ctypes.c_void_p(4096)
    # missing pointers, bad scale, short or misaligned workspace: before any device work
    assert L.gftorf_mlp_forward(10, 2, None, 256, t, 0.2, 256, ws, small, None) == gftorf.ERR_ARG
    assert L.gftorf_mlp_forward(10, 2, 256, 256, t, 0.0, 256, ws, small, None) == gftorf.ERR_ARG
    assert L.gftorf_mlp_forward(1000, 2, 256, 256, t, 0.2, 256, ws, small - 1,
                                None) == gftorf.ERR_WORKSPACE
    assert L.gftorf_mlp_forward(1000, 2, 256, 256, t, 0.2, 256, ctypes.c_void_p(4100), small,
                                None) == gftorf.ERR_WORKSPACE
    t[1] = float("nan")
    assert L.gftorf_mlp_forward(1000, 2, 256, 256, t, 0.2, 256, ws, small,
                                None) == gftorf.ERR_ARG
    assert L.gftorf_mlp_backward(10, 2, 256, 256, t, 0.2, None, 256, 256, ws, small,
                                 None) == gftorf.ERR_ARG
    assert L.gftorf_mlp_export(1000, 2, 9, 0, 256, ws, small, None) == gftorf.ERR_ARG
    assert L.gftorf_mlp_export(1000, 2, 1, 8, 256, ws, small, None) == gftorf.ERR_ARG


def test_throughput_probe_rejects_bad_arguments_on_host(lib):
    ops = ctypes.c_int64(0)
    fake = ctypes.c_void_p(256)  # never dereferenced: every call below fails its host checks
    for kind, iters in ((2, 64), (-1, 64), (0, 0), (0, 17), (1, -16)):
        assert lib.gftorf_probe_throughput(kind, iters, fake, ctypes.byref(ops), None) == \
            gftorf.ERR_ARG, (kind, iters)
    assert lib.gftorf_probe_throughput(0, 64, None, ctypes.byref(ops), None) == gftorf.ERR_ARG
    assert lib.gftorf_probe_throughput(0, 64, fake, None, None) == gftorf.ERR_ARG
