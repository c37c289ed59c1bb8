"""Thin ctypes binding of libgftorf.so (include/gftorf.h), same names.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels; PyTorch provides device memory (workspace, outputs) and the stream.
Loading fails loudly when the library is missing or no CUDA device exists.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Dict, List, Optional, Sequence, Tuple

import torch

from . import build as _build

# --- mirrors of include/gftorf.h -------------------------------------------
MAX_FREQ, MAX_OFFSETS, MAX_FRAMES = 4, 8, 64
F32, F64 = 0, 1
STATUS = {0: "ok", 1: "invalid argument", 2: "tile-instance capacity exceeded",
          3: "bounded device wait timed out", 4: "CUDA error",
          5: "unsupported configuration", 6: "workspace missing, misaligned or too small"}
OK, ERR_ARG, ERR_CAPACITY, ERR_TIMEOUT, ERR_CUDA, ERR_UNSUPPORTED, ERR_WORKSPACE = range(7)
FLAG_NO_TILE_CULL = 1
FLAG_COUNT_PAIRS = 2
FLAG_PHASOR = 4
FLAG_DEPTH = 8


class Dims(ctypes.Structure):
    _fields_ = [("n_gaussians", ctypes.c_int32), ("n_frames", ctypes.c_int32),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("n_freq", ctypes.c_int32), ("n_offsets", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("render_mode", ctypes.c_int32),
                ("pixels_per_thread", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("n_sh", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("max_instances", ctypes.c_int64)]


class Frame(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("world_to_cam", ctypes.c_float * 12),
                ("near_plane", ctypes.c_float), ("time", ctypes.c_float),
                ("phase_offset_rad", ctypes.c_float), ("interp_t0", ctypes.c_float),
                ("interp_t1", ctypes.c_float)]


class Sensor(ctypes.Structure):
    _fields_ = [("freq_hz", ctypes.c_float * MAX_FREQ),
                ("offset_rad", ctypes.c_float * MAX_OFFSETS),
                ("source_intensity", ctypes.c_float)]


class Consts(ctypes.Structure):
    _fields_ = [("dilation", ctypes.c_float), ("alpha_max", ctypes.c_float),
                ("alpha_min", ctypes.c_float), ("t_min", ctypes.c_float),
                ("guard", ctypes.c_float), ("sigma_cut", ctypes.c_float)]


class Gaussians(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in
                ("means", "coeffs", "scales", "quats", "opacity", "amplitude", "delta", "sh")]


class AdamGroup(ctypes.Structure):
    _fields_ = [("param", ctypes.c_void_p), ("grad", ctypes.c_void_p), ("m", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("n", ctypes.c_int64), ("lr", ctypes.c_float),
                ("lo", ctypes.c_float), ("hi", ctypes.c_float)]


MAX_ADAM_GROUPS = 12


class Gradients(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in
                ("means", "coeffs", "scales", "quats", "opacity", "amplitude", "delta", "bg",
                 "sh")]


_LIB = None
_P = ctypes.POINTER


def kernel_launches() -> int:
    """Kernels the library has enqueued in this process so far."""
    return int(load().gftorf_kernel_launches())


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgftorf.so (building it in-tree first if needed)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libgftorf.so is missing (%s); run build()" % path)
    L = ctypes.CDLL(path)
    vp, sz = ctypes.c_void_p, ctypes.c_size_t
    L.gftorf_version.restype = ctypes.c_int32
    L.gftorf_status_string.restype = ctypes.c_char_p
    L.gftorf_status_string.argtypes = [ctypes.c_int]
    L.gftorf_workspace_size.restype = sz
    L.gftorf_workspace_size.argtypes = [_P(Dims)]
    L.gftorf_preprocess.argtypes = [_P(Dims), _P(Gaussians), _P(Frame), _P(Sensor),
                                    _P(Consts), vp, sz, vp]
    L.gftorf_render_fwd.argtypes = [_P(Dims), vp, vp, vp, sz, vp]
    L.gftorf_render_bwd.argtypes = [_P(Dims), _P(Gaussians), vp, vp, _P(Gradients), vp, sz, vp]
    L.gftorf_sort_footprints.argtypes = [_P(Dims), vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    L.gftorf_export_tile_lists.argtypes = [_P(Dims), vp, vp, vp, vp, vp, sz, vp]
    L.gftorf_export_pixel_state.argtypes = [_P(Dims), vp, vp, vp, sz, vp]
    L.gftorf_read_device_status.argtypes = [_P(Dims), vp, sz, _P(ctypes.c_int64), vp]
    L.gftorf_bin.argtypes = [_P(Dims), vp, sz, vp]
    L.gftorf_composite_fwd.argtypes = [_P(Dims), vp, vp, vp, sz, vp]
    L.gftorf_zero_grad_buffers.argtypes = [_P(Dims), _P(Gradients), vp, sz, vp]
    L.gftorf_composite_bwd.argtypes = [_P(Dims), vp, vp, _P(Gradients), vp, sz, vp]
    L.gftorf_preprocess_bwd.argtypes = [_P(Dims), _P(Gaussians), _P(Gradients), vp, sz, vp]
    L.gftorf_sort_footprints_noalloc.argtypes = [_P(Dims), vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.gftorf_sort_footprints_noalloc.restype = ctypes.c_int
    L.gftorf_read_counters.argtypes = [_P(Dims), vp, sz, _P(ctypes.c_int64), vp]
    L.gftorf_read_counters.restype = ctypes.c_int
    L.gftorf_kernel_launches.restype = ctypes.c_int64
    L.gftorf_kernel_launches.argtypes = []
    L.gftorf_probe_throughput.argtypes = [ctypes.c_int32, ctypes.c_int32, vp,
                                          _P(ctypes.c_int64), vp]
    L.gftorf_probe_throughput.restype = ctypes.c_int
    L.gftorf_train_begin.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_uint64, vp]
    L.gftorf_train_begin_shard.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_uint64,
                                           ctypes.c_int64, ctypes.c_int64, vp]
    L.gftorf_l2_loss.argtypes = [_P(Dims), vp, vp, vp, vp, vp]
    L.gftorf_l2_loss_scaled.argtypes = [_P(Dims), vp, vp, vp, vp, ctypes.c_double, vp]
    L.gftorf_adam_step.argtypes = [_P(AdamGroup), ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_float, vp, vp]
    for name in ("gftorf_preprocess", "gftorf_render_fwd", "gftorf_render_bwd",
                 "gftorf_sort_footprints", "gftorf_export_tile_lists",
                 "gftorf_export_pixel_state", "gftorf_read_device_status",
                 "gftorf_bin", "gftorf_composite_fwd", "gftorf_zero_grad_buffers",
                 "gftorf_composite_bwd", "gftorf_preprocess_bwd", "gftorf_train_begin",
                 "gftorf_train_begin_shard", "gftorf_l2_loss", "gftorf_l2_loss_scaled",
                 "gftorf_adam_step"):
        getattr(L, name).restype = ctypes.c_int
    _LIB = L
    return L


class GftorfError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("%s: %s (status %d)" % (what, STATUS.get(code, "?"), code))
        self.code = code


def _check(code: int, what: str):
    if code != OK:
        raise GftorfError(code, what)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("gftorf needs a CUDA device; none is available")


# --- argument builders -------------------------------------------------------
def make_frame(fx, fy, cx, cy, world_to_cam, near_plane, time, phase_offset_rad=0.0,
               interp=None) -> Frame:
    """interp = (t0, t1): Eq. 7 interpolation of the positions between two
    timesteps; phase_offset_rad: this frame's own phase offset (asynchronous
    raw capture)."""
    f = Frame()
    f.fx, f.fy, f.cx, f.cy = fx, fy, cx, cy
    wc = [float(v) for v in torch.as_tensor(world_to_cam, dtype=torch.float64).reshape(12)]
    for i in range(12):
        f.world_to_cam[i] = wc[i]
    f.near_plane, f.time = near_plane, time
    f.phase_offset_rad = phase_offset_rad
    if interp is not None:
        f.interp_t0, f.interp_t1 = float(interp[0]), float(interp[1])
    return f


def make_sensor(freqs_hz: Sequence[float], offsets_rad: Sequence[float],
                source_intensity: float = 1.0) -> Sensor:
    s = Sensor()
    for i, v in enumerate(freqs_hz):
        s.freq_hz[i] = v
    for i, v in enumerate(offsets_rad):
        s.offset_rad[i] = v
    s.source_intensity = source_intensity
    return s


def make_consts(dilation=0.3, alpha_max=0.99, alpha_min=1.0 / 255.0, t_min=1e-4,
                guard=1.3, sigma_cut=3.0) -> Consts:
    c = Consts()
    c.dilation, c.alpha_max, c.alpha_min = dilation, alpha_max, alpha_min
    c.t_min, c.guard, c.sigma_cut = t_min, guard, sigma_cut
    return c


def frames_from_scene(scene) -> List[Frame]:
    out = []
    ph = getattr(scene, "frame_phase", None)
    it = getattr(scene, "interp_times", None)
    for b, cam in enumerate(scene.cameras):
        out.append(make_frame(cam.fx, cam.fy, cam.cx, cam.cy, cam.world_to_cam,
                              cam.near, float(scene.times[b]),
                              0.0 if ph is None else float(ph[b]),
                              None if it is None else it[b]))
    return out


def sensor_from_scene(scene) -> Sensor:
    s = scene.sensor
    return make_sensor(s.freqs_hz, s.offsets_rad, s.source_intensity)


def flags_from_scene(scene) -> int:
    """Output-channel flags a scene's constants ask for."""
    k = scene.consts
    return ((FLAG_PHASOR if getattr(k, "phasor", False) else 0) |
            (FLAG_DEPTH if getattr(k, "depth", False) else 0))


def consts_from_scene(scene) -> Consts:
    k = scene.consts
    return make_consts(k.dilation, k.alpha_max, k.alpha_min, k.t_min, k.guard, k.sigma_cut)


PARAM_NAMES = ("means", "coeffs", "scales", "quats", "opacity", "amplitude", "delta", "sh")
GRAD_NAMES = ("means", "coeffs", "scales", "quats", "opacity", "amplitude", "delta", "bg", "sh")


def params_from_scene(scene, device="cuda", dtype=torch.float32) -> Dict[str, torch.Tensor]:
    """Scene arrays as device tensors (coeffs / delta / sh may be None)."""
    out = {}
    for k in PARAM_NAMES:
        a = getattr(scene, k, None)
        out[k] = None if a is None else torch.as_tensor(a).to(device=device, dtype=dtype).contiguous()
    return out


# --- workspace + calls ---------------------------------------------------------
class Renderer:
    """One workspace for a fixed problem shape; wraps the C ABI calls.

    The library never allocates: the workspace is a torch uint8 tensor sized
    by gftorf_workspace_size.  All calls enqueue on torch's current stream.
    """

    def __init__(self, n, frames, width, height, n_freq=1, n_offsets=4,
                 tile=(16, 16), dtype=torch.float32, render_mode=0,
                 max_instances=None, device="cuda", pixels_per_thread=0, flags=0, n_sh=0):
        _require_cuda()
        self.lib = load()
        self.torch_dtype = dtype
        self.device = torch.device(device)
        self.dims = Dims(n, frames, width, height, tile[0], tile[1], n_freq,
                         n_offsets, F64 if dtype == torch.float64 else F32,
                         render_mode, pixels_per_thread, flags, n_sh, 0, 0)
        self.C = (n_freq * n_offsets + 1 + (2 * n_freq if flags & FLAG_PHASOR else 0) +
                  (1 if flags & FLAG_DEPTH else 0))
        self.tiles_x = -(-width // tile[0])
        self.tiles_y = -(-height // tile[1])
        self.n_tiles = self.tiles_x * self.tiles_y
        self._set_capacity(max_instances if max_instances is not None else max(1, 16 * n * frames))

    def _set_capacity(self, cap: int):
        self.dims.max_instances = int(cap)
        nbytes = self.lib.gftorf_workspace_size(ctypes.byref(self.dims))
        if nbytes == 0:
            raise GftorfError(ERR_ARG, "gftorf_workspace_size")
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        off = (-self.ws.data_ptr()) % 256
        self.ws_ptr = ctypes.c_void_p(self.ws.data_ptr() + off)
        self.ws_bytes = nbytes

    @property
    def capacity(self) -> int:
        return int(self.dims.max_instances)

    def _gaussians(self, p: Dict[str, torch.Tensor]) -> Gaussians:
        nsh = self.dims.n_sh
        sh = p.get("sh")
        if nsh and (sh is None or sh.dim() != 2 or sh.shape[1] != nsh):
            raise ValueError("sh must be (N, %d) for n_sh = %d" % (nsh, nsh))
        g = Gaussians()
        for k in PARAM_NAMES:
            t = p.get(k)
            if t is not None:
                if t.dtype != self.torch_dtype:
                    raise ValueError("%s has dtype %s, expected %s" % (k, t.dtype, self.torch_dtype))
                setattr(g, k, _ptr(t))
        return g

    generation = 0  # bumped by every preprocess: identifies the workspace's batch

    def preprocess(self, params, frames: Sequence[Frame], sensor: Sensor, consts: Consts):
        arr = (Frame * len(frames))(*frames)
        self._keep = (params, arr)
        self.generation += 1
        _check(self.lib.gftorf_preprocess(ctypes.byref(self.dims),
                                          ctypes.byref(self._gaussians(params)), arr,
                                          ctypes.byref(sensor), ctypes.byref(consts),
                                          self.ws_ptr, self.ws_bytes, _stream()),
               "gftorf_preprocess")

    def render_fwd(self, bg: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        d = self.dims
        if out is None:
            out = torch.empty((d.n_frames, self.C, d.height, d.width),
                              dtype=self.torch_dtype, device=self.device)
        _check(self.lib.gftorf_render_fwd(ctypes.byref(d), _ptr(bg), _ptr(out),
                                          self.ws_ptr, self.ws_bytes, _stream()),
               "gftorf_render_fwd")
        return out

    def render_bwd(self, params, bg, dout, grads: Optional[Dict[str, torch.Tensor]] = None,
                   want=GRAD_NAMES):
        d = self.dims
        if grads is None:
            grads = self.alloc_grads(params, bg, want)
        gr = self._grad_struct(grads)
        _check(self.lib.gftorf_render_bwd(ctypes.byref(d), ctypes.byref(self._gaussians(params)),
                                          _ptr(bg), _ptr(dout), ctypes.byref(gr),
                                          self.ws_ptr, self.ws_bytes, _stream()),
               "gftorf_render_bwd")
        return grads

    # --- the stages, one by one ------------------------------------------------
    def bin(self):
        _check(self.lib.gftorf_bin(ctypes.byref(self.dims), self.ws_ptr, self.ws_bytes,
                                   _stream()), "gftorf_bin")

    def composite_fwd(self, bg, out):
        _check(self.lib.gftorf_composite_fwd(ctypes.byref(self.dims), _ptr(bg), _ptr(out),
                                             self.ws_ptr, self.ws_bytes, _stream()),
               "gftorf_composite_fwd")
        return out

    def _grad_struct(self, grads):
        gr = Gradients()
        for k, t in grads.items():
            setattr(gr, k, _ptr(t))
        return gr

    def zero_grad_buffers(self, grads):
        _check(self.lib.gftorf_zero_grad_buffers(ctypes.byref(self.dims),
                                                 ctypes.byref(self._grad_struct(grads)),
                                                 self.ws_ptr, self.ws_bytes, _stream()),
               "gftorf_zero_grad_buffers")

    def composite_bwd(self, bg, dout, grads):
        _check(self.lib.gftorf_composite_bwd(ctypes.byref(self.dims), _ptr(bg), _ptr(dout),
                                             ctypes.byref(self._grad_struct(grads)),
                                             self.ws_ptr, self.ws_bytes, _stream()),
               "gftorf_composite_bwd")

    def preprocess_bwd(self, params, grads):
        _check(self.lib.gftorf_preprocess_bwd(ctypes.byref(self.dims),
                                              ctypes.byref(self._gaussians(params)),
                                              ctypes.byref(self._grad_struct(grads)),
                                              self.ws_ptr, self.ws_bytes, _stream()),
               "gftorf_preprocess_bwd")

    def alloc_grads(self, params, bg, want=GRAD_NAMES):
        grads = {}
        for k in want:
            if k == "bg":
                grads[k] = torch.empty_like(bg)
            elif params.get(k) is not None:
                grads[k] = torch.empty_like(params[k])
        return grads

    def read_status(self):
        """(status code, instance count); synchronises the stream."""
        cnt = ctypes.c_int64(0)
        code = self.lib.gftorf_read_device_status(ctypes.byref(self.dims), self.ws_ptr,
                                                  self.ws_bytes, ctypes.byref(cnt), _stream())
        return code, int(cnt.value)

    def counters(self, with_warp=False):
        """(instances, evaluated pairs) of the last binning / forward, and with
        with_warp the evaluated pairs in records that reach the pixel's warp;
        pairs are counted only with FLAG_COUNT_PAIRS.  Synchronises."""
        buf = (ctypes.c_int64 * 3)()
        _check(self.lib.gftorf_read_counters(ctypes.byref(self.dims), self.ws_ptr, self.ws_bytes,
                                             buf, _stream()), "gftorf_read_counters")
        if with_warp:
            return int(buf[0]), int(buf[1]), int(buf[2])
        return int(buf[0]), int(buf[1])

    def check(self):
        code, cnt = self.read_status()
        _check(code, "device status")
        return cnt

    def tile_lists(self, with_keys=True):
        """(keys u64 | None, values u32, ranges (B*tiles, 2), count) on device."""
        d = self.dims
        cap = max(self.capacity, 1)
        vals = torch.empty(cap, dtype=torch.int32, device=self.device)
        keys = torch.empty(cap, dtype=torch.int64, device=self.device) if with_keys else None
        ranges = torch.empty((d.n_frames * self.n_tiles, 2), dtype=torch.int32, device=self.device)
        count = torch.zeros(1, dtype=torch.int64, device=self.device)
        _check(self.lib.gftorf_export_tile_lists(ctypes.byref(d), _ptr(keys), _ptr(vals),
                                                 _ptr(ranges), _ptr(count), self.ws_ptr,
                                                 self.ws_bytes, _stream()),
               "gftorf_export_tile_lists")
        return keys, vals, ranges, count

    def pixel_state(self):
        d = self.dims
        tf = torch.empty((d.n_frames, d.height, d.width), dtype=self.torch_dtype, device=self.device)
        nl = torch.empty((d.n_frames, d.height, d.width), dtype=torch.int32, device=self.device)
        _check(self.lib.gftorf_export_pixel_state(ctypes.byref(d), _ptr(tf), _ptr(nl),
                                                  self.ws_ptr, self.ws_bytes, _stream()),
               "gftorf_export_pixel_state")
        return tf, nl

    def fit_capacity(self, params, frames, sensor, consts, bg, headroom=1.15):
        """Run preprocess + binning once, read the instance count and resize
        the workspace to hold it (synchronises; not for use inside capture)."""
        self.preprocess(params, frames, sensor, consts)
        self.render_fwd(bg)
        code, cnt = self.read_status()
        if code not in (OK, ERR_CAPACITY):
            _check(code, "device status")
        need = max(1, int(math.ceil(cnt * headroom)) + 1024)
        if need > self.capacity or code == ERR_CAPACITY:
            self._set_capacity(need)
        return cnt


def sort_footprints(u, v, radius, z, width, height, tile=(16, 16), max_instances=None):
    """Binning alone from float32 footprints shaped (B, N) (device tensors).
    Returns (keys int64 (M,), values int32 (M,), ranges int32 (B*tiles, 2))."""
    _require_cuda()
    L = load()
    B, n = u.shape
    if max_instances is None:
        r = radius.to(torch.int64).clamp(min=0)
        max_instances = int((((2 * r) // tile[0] + 2) * ((2 * r) // tile[1] + 2)).sum().item())
    dims = Dims(n, B, width, height, tile[0], tile[1], 1, 1, F32, 0, 0, 0,
                max_instances=max(1, max_instances))
    nbytes = L.gftorf_workspace_size(ctypes.byref(dims))
    if nbytes == 0:
        raise GftorfError(ERR_ARG, "gftorf_workspace_size")
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=u.device)
    off = (-ws.data_ptr()) % 256
    cap = max(1, max_instances)
    keys = torch.empty(cap, dtype=torch.int64, device=u.device)
    vals = torch.empty(cap, dtype=torch.int32, device=u.device)
    tiles = (-(-width // tile[0])) * (-(-height // tile[1]))
    ranges = torch.empty((B * tiles, 2), dtype=torch.int32, device=u.device)
    count = torch.zeros(1, dtype=torch.int64, device=u.device)
    _check(L.gftorf_sort_footprints(ctypes.byref(dims), _ptr(u), _ptr(v), _ptr(radius), _ptr(z),
                                    _ptr(keys), _ptr(vals), _ptr(ranges), _ptr(count),
                                    ctypes.c_void_p(ws.data_ptr() + off), nbytes, _stream()),
           "gftorf_sort_footprints")
    cnt = ctypes.c_int64(0)
    code = L.gftorf_read_device_status(ctypes.byref(dims), ctypes.c_void_p(ws.data_ptr() + off),
                                       nbytes, ctypes.byref(cnt), _stream())
    _check(code, "device status")
    m = int(cnt.value)
    return keys[:m], vals[:m], ranges


def sort_footprints_noalloc(u, v, radius, z, width, height, tile=(16, 16), max_instances=1):
    """gftorf_sort_footprints_noalloc: the same binning with the library's
    fixed device scratch (no workspace).  Output buffers are allocated here by
    torch for convenience; the entry point itself allocates nothing.
    Returns (status, keys, values, ranges, count_tensor)."""
    _require_cuda()
    L = load()
    B, n = u.shape
    dims = Dims(n, B, width, height, tile[0], tile[1], 1, 1, F32, 0, 0, 0,
                max_instances=int(max_instances))
    cap = max(1, int(max_instances))
    keys = torch.empty(cap, dtype=torch.int64, device=u.device)
    vals = torch.empty(cap, dtype=torch.int32, device=u.device)
    tiles = (-(-width // tile[0])) * (-(-height // tile[1]))
    ranges = torch.empty((B * tiles, 2), dtype=torch.int32, device=u.device)
    count = torch.zeros(1, dtype=torch.int64, device=u.device)
    code = L.gftorf_sort_footprints_noalloc(ctypes.byref(dims), _ptr(u), _ptr(v), _ptr(radius),
                                            _ptr(z), _ptr(keys), _ptr(vals), _ptr(ranges),
                                            _ptr(count), _stream())
    return code, keys, vals, ranges, count


PROBE_FFMA, PROBE_EX2 = 0, 1


def probe_throughput(kind: int, iters: int, sink: torch.Tensor) -> int:
    """gftorf_probe_throughput: enqueue one throughput-probe launch on the
    current stream; returns the lane operations it performs."""
    ops = ctypes.c_int64(0)
    _check(load().gftorf_probe_throughput(int(kind), int(iters), _ptr(sink), ctypes.byref(ops),
                                          _stream()), "gftorf_probe_throughput")
    return int(ops.value)


def measure_alu_peaks(iters: int = 4096, reps: int = 5) -> Dict[str, float]:
    """FP32 FMA and ex2 lane operations per second of this device (best of
    `reps` launches, CUDA events on the current stream, after a warm-up)."""
    sink = torch.zeros(1, device="cuda")
    out = {}
    for name, kind in (("ffma", PROBE_FFMA), ("ex2", PROBE_EX2)):
        probe_throughput(kind, iters, sink)
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ops = probe_throughput(kind, iters, sink)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        out[name] = ops / (best / 1e3)
        out[name + "_ms"] = best
    return out


# --- autograd ------------------------------------------------------------------
class RenderCToF(torch.autograd.Function):
    """Raw C-ToF render of a batch of frames, differentiable w.r.t. the
    Gaussian parameters, the per-frame displacement and the background.

    forward(renderer, frames, sensor, consts, bg, means, coeffs, scales, quats,
            opacity, amplitude, delta, sh) -> out[B][C][H][W]
    (coeffs, delta, sh may be None; amplitude is unused when sh is given)
    """

    @staticmethod
    def forward(ctx, renderer: Renderer, frames, sensor, consts, bg, means, coeffs,
                scales, quats, opacity, amplitude, delta, sh=None):
        c = lambda t: None if t is None else t.contiguous()
        params = dict(means=means.contiguous(), coeffs=c(coeffs),
                      scales=scales.contiguous(), quats=quats.contiguous(),
                      opacity=opacity.contiguous(), amplitude=c(amplitude),
                      delta=c(delta), sh=c(sh))
        renderer.preprocess(params, frames, sensor, consts)
        out = renderer.render_fwd(bg.contiguous())
        ctx.renderer = renderer
        ctx.params = params
        ctx.setup = (frames, sensor, consts)
        ctx.generation = renderer.generation
        ctx.save_for_backward(bg)
        return out

    @staticmethod
    def backward(ctx, dout):
        (bg,) = ctx.saved_tensors
        r, p = ctx.renderer, ctx.params
        if r.generation != ctx.generation:
            # the workspace now holds another batch: recompute this one
            r.preprocess(p, *ctx.setup)
            r.render_fwd(bg.contiguous())
        want = ["means", "scales", "quats", "opacity", "bg"]
        for k in ("amplitude", "coeffs", "delta", "sh"):
            if p[k] is not None:
                want.append(k)
        g = r.render_bwd(p, bg.contiguous(), dout.contiguous(), want=want)
        return (None, None, None, None, g.get("bg"), g.get("means"), g.get("coeffs"),
                g.get("scales"), g.get("quats"), g.get("opacity"), g.get("amplitude"),
                g.get("delta"), g.get("sh"))


def render_ctof(renderer, frames, sensor, consts, bg, params):
    return RenderCToF.apply(renderer, frames, sensor, consts, bg, params["means"],
                            params.get("coeffs"), params["scales"], params["quats"],
                            params["opacity"], params.get("amplitude"), params.get("delta"),
                            params.get("sh"))


# --- optimisation loop ---------------------------------------------------------
def new_train_state(device="cuda") -> torch.Tensor:
    """Zeroed gftorf_train_state (32 bytes) on the device."""
    return torch.zeros(4, dtype=torch.int64, device=device)


def train_step_count(state: torch.Tensor) -> int:
    return int(state[0].item())


def train_loss(state: torch.Tensor) -> float:
    """The current iteration's loss (synchronises)."""
    return float(state.view(torch.float64)[1].item())


def train_begin(state: torch.Tensor, bg: Optional[torch.Tensor], seed: int,
                bg_offset: int = 0, bg_stride: Optional[int] = None):
    """Device-side iteration start: step += 1, loss = 0, fresh random bg.
    With bg_offset / bg_stride (a shard of a batch's frames): bg gets values
    [bg_offset, bg_offset + bg.numel()) of the batch's bg_stride values."""
    L = load()
    n = 0 if bg is None else bg.numel()
    if bg is not None and (bg.dtype != torch.float32 or not bg.is_contiguous()):
        raise ValueError("bg must be contiguous float32")
    stride = n if bg_stride is None else int(bg_stride)
    _check(L.gftorf_train_begin_shard(_ptr(state), _ptr(bg), n, seed & ((1 << 64) - 1),
                                      int(bg_offset), stride, _stream()),
           "gftorf_train_begin")


def l2_loss(renderer: "Renderer", out, target, dout, state, count: Optional[float] = None):
    """dL/dout of the raw-sample L2 loss (written into dout); adds L to the
    state's loss.  count: the number of raw samples the mean is over (default:
    this batch's; a shard of frames passes the whole batch's)."""
    if count is None:
        code = renderer.lib.gftorf_l2_loss(ctypes.byref(renderer.dims), _ptr(out), _ptr(target),
                                           _ptr(dout), _ptr(state), _stream())
    else:
        code = renderer.lib.gftorf_l2_loss_scaled(ctypes.byref(renderer.dims), _ptr(out),
                                                  _ptr(target), _ptr(dout), _ptr(state),
                                                  float(count), _stream())
    _check(code, "gftorf_l2_loss")


class Adam:
    """Fused projected Adam over named parameter tensors (one launch).

    lrs: name -> learning rate; bounds: name -> (lo, hi).  Moments live here;
    the step count comes from the device-side train state."""

    def __init__(self, params: Dict[str, torch.Tensor], lrs: Dict[str, float],
                 bounds: Optional[Dict[str, Tuple[float, float]]] = None,
                 betas=(0.9, 0.999), eps=1e-15):
        self.lib = load()
        self.names = [k for k in lrs if params.get(k) is not None]
        if len(self.names) > MAX_ADAM_GROUPS:
            raise ValueError("at most %d parameter groups" % MAX_ADAM_GROUPS)
        self.params = params
        self.m = {k: torch.zeros_like(params[k]) for k in self.names}
        self.v = {k: torch.zeros_like(params[k]) for k in self.names}
        self.lrs = dict(lrs)
        self.bounds = dict(bounds or {})
        self.betas, self.eps = betas, eps

    def _groups(self, grads):
        arr = (AdamGroup * len(self.names))()
        for i, k in enumerate(self.names):
            p, g = self.params[k], grads[k]
            if (p.dtype != torch.float32 or g.dtype != torch.float32 or g.shape != p.shape
                    or not p.is_contiguous() or not g.is_contiguous()):
                raise ValueError("group %s: contiguous float32 param and grad of the same "
                                 "shape required" % k)
            lo, hi = self.bounds.get(k, (-math.inf, math.inf))
            arr[i] = AdamGroup(_ptr(p), _ptr(g), _ptr(self.m[k]), _ptr(self.v[k]), p.numel(),
                               self.lrs[k], lo, hi)
        return arr

    def step(self, grads: Dict[str, torch.Tensor], state: torch.Tensor):
        arr = self._groups(grads)
        self._keep = arr
        _check(self.lib.gftorf_adam_step(arr, len(self.names), self.betas[0], self.betas[1],
                                         self.eps, _ptr(state), _stream()),
               "gftorf_adam_step")
