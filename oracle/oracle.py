"""ctypes front end of the FP64 oracle library (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It never imports the CUDA package: it
reads the scene's arrays by attribute and widens them to float64.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build_oracle

_LIB = None

# packed layouts (gftorf_oracle.h)
MAX_F, MAX_P = 4, 8
FR_LEN = 23
SE_LEN = 1 + MAX_F + 1 + MAX_P + 1
CO_LEN = 11
MAX_SH = 16
NPARAM = 24 + MAX_SH
SP = dict(VIS=0, U=1, V=2, CA=3, CB=4, CC=5, OPA=6, Z=7, D=8, RAD=9,
          X0=10, Y0=11, X1=12, Y1=13, MX0=14, MY0=15, MX1=16, MY1=17,
          IX0=18, IY0=19, IX1=20, IY1=21, UNCERT=22, AMP=23, FEAT=24)
AMB = dict(ALPHA_MIN=1, TMIN=2, ORDER=4, CLAMP=8, RECT=16, POWER=32)
# value-changing flags (the clamp flag only affects gradients)
AMB_VALUE = AMB["ALPHA_MIN"] | AMB["TMIN"] | AMB["ORDER"] | AMB["RECT"] | AMB["POWER"]

# margins: a single-precision implementation may decide the other way when the
# oracle's value lies this close to a threshold (relative).  The alpha margin
# covers the FP32 exponent argument error (|power| ~ 5 at the 1/255 threshold),
# the T margin is per composited step, the depth margin a few FP32 ulps (a
# depth computed in single precision as a short sum of products is within
# ~2 ulps of the exact one, so two depths closer than ~4 ulps may swap).
EPS_F32 = (2e-5, 4e-6, 6e-7, 2e-5)
EPS_F64 = (1e-10, 1e-11, 1e-11, 1e-10)
EPS_NONE = (0.0, 0.0, 0.0, 0.0)

_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_f32 = ctypes.POINTER(ctypes.c_float)
_u64 = ctypes.POINTER(ctypes.c_uint64)
_u32 = ctypes.POINTER(ctypes.c_uint32)


def lib():
    global _LIB
    if _LIB is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        L.ora_splat_len.restype = ctypes.c_int
        L.ora_num_threads.restype = ctypes.c_int
        L.ora_set_threads.argtypes = [ctypes.c_int]
        L.ora_project.argtypes = [ctypes.c_int] + [_d] * 13
        L.ora_sh_basis.argtypes = [ctypes.c_int] + [ctypes.c_double] * 3
        L.ora_sh_basis.restype = ctypes.c_double
        L.ora_render_pixels.argtypes = [ctypes.c_int, _d, _d, _d, _d, _d, _d,
                                        ctypes.c_int, _i32, _d, _d, _i32, _i32]
        L.ora_pixel_steps.argtypes = [ctypes.c_int, _d, _d, _d, _d, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, _d, _d, _d]
        L.ora_pixel_steps.restype = ctypes.c_int
        L.ora_render_frame.argtypes = [ctypes.c_int, _d, _d, _d, _d, _d, _d,
                                       _d, _d, _i32, _i32]
        L.ora_backward_2d.argtypes = [ctypes.c_int, _d, _d, _d, _d, _d, _d, _d, _d]
        L.ora_backward_params.argtypes = [ctypes.c_int] + [_d] * 14
        _i64 = ctypes.POINTER(ctypes.c_int64)
        L.ora_render_tiles.argtypes = [ctypes.c_int, _d, _d, _d, _d, _d, _d, ctypes.c_int, _i32,
                                       _d, _d, _i32, _i32, ctypes.c_int, ctypes.c_int64, _d,
                                       _i64, _i64, _i64]
        L.ora_render_tiles.restype = ctypes.c_int64
        L.ora_bin_f32.argtypes = [ctypes.c_int, ctypes.c_int, _f32, _f32, _i32,
                                  _f32, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int64, _u64, _u32, _u32]
        L.ora_bin_f32.restype = ctypes.c_int64
        assert L.ora_splat_len() == SP["FEAT"] + 2 * MAX_F + 1
        _LIB = L
    return _LIB


def num_threads() -> int:
    return lib().ora_num_threads()


def set_threads(n: int):
    """OpenMP threads of the oracle's following calls."""
    lib().ora_set_threads(int(n))


def _p(a, t=_d):
    if a is None:
        return None
    return a.ctypes.data_as(t)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def pack_frame(scene, b: int) -> np.ndarray:
    cam = scene.cameras[b]
    fr = np.zeros(FR_LEN)
    fr[0:6] = [cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy]
    fr[6:18] = np.asarray(cam.world_to_cam, np.float64).reshape(12)
    fr[18] = cam.near
    fr[19] = float(scene.times[b])
    ph = getattr(scene, "frame_phase", None)
    fr[20] = 0.0 if ph is None else float(ph[b])
    it = getattr(scene, "interp_times", None)
    if it is not None:
        fr[21], fr[22] = float(it[b][0]), float(it[b][1])
    return fr


def pack_sensor(scene) -> np.ndarray:
    s = scene.sensor
    se = np.zeros(SE_LEN)
    se[0] = len(s.freqs_hz)
    se[1:1 + len(s.freqs_hz)] = s.freqs_hz
    se[1 + MAX_F] = len(s.offsets_rad)
    se[2 + MAX_F:2 + MAX_F + len(s.offsets_rad)] = s.offsets_rad
    se[2 + MAX_F + MAX_P] = s.source_intensity
    return se


def pack_consts(scene) -> np.ndarray:
    k = scene.consts
    return np.array([k.dilation, k.alpha_max, k.alpha_min, k.t_min, k.guard,
                     k.sigma_cut, k.tile_w, k.tile_h, float(getattr(k, "phasor", False)),
                     float(getattr(k, "depth", False)), float(n_sh(scene))], np.float64)


def n_sh(scene) -> int:
    """SH coefficients per Gaussian (0: scalar reflectivity)."""
    sh = getattr(scene, "sh", None)
    return 0 if sh is None else int(np.asarray(sh).shape[1])


def sh_basis(l: int, x: float, y: float, z: float) -> float:
    """Real SH basis function l (degree-major, 0..15) at a unit vector."""
    return lib().ora_sh_basis(l, x, y, z)


def n_channels(scene) -> int:
    """Output channels: F*P raw + ambient (+ 2F phasor) (+ depth)."""
    F = len(scene.sensor.freqs_hz)
    k = scene.consts
    return (F * len(scene.sensor.offsets_rad) + 1 + (2 * F if getattr(k, "phasor", False) else 0)
            + (1 if getattr(k, "depth", False) else 0))


def _copy64(a):
    return np.array(a, dtype=np.float64, copy=True, order="C")


class Params:
    """float64 copies of a scene's Gaussian parameters (optionally replaced)."""

    def __init__(self, scene, **over):
        self.means = _copy64(over.get("means", scene.means))
        co = over.get("coeffs", scene.coeffs)
        self.coeffs = _copy64(co) if co is not None else np.zeros((scene.n, 3, 3))
        self.scales = _copy64(over.get("scales", scene.scales))
        self.quats = _copy64(over.get("quats", scene.quats))
        self.opacity = _copy64(over.get("opacity", scene.opacity))
        self.amplitude = _copy64(over.get("amplitude", scene.amplitude))
        de = over.get("delta", scene.delta)
        self.delta = _copy64(de) if de is not None else None
        sh = over.get("sh", getattr(scene, "sh", None))
        self.sh = None
        if sh is not None:
            sh = np.asarray(sh, np.float64)
            self.sh = np.zeros((scene.n, MAX_SH))
            self.sh[:, :sh.shape[1]] = sh

    def delta_of(self, b):
        return None if self.delta is None else np.ascontiguousarray(self.delta[b])


def project(scene, b: int, eps=EPS_NONE, params: Params = None) -> np.ndarray:
    """Splat records (N, SP_LEN) of frame b."""
    P = params or Params(scene)
    n = scene.n
    out = np.zeros((n, lib().ora_splat_len()))
    e = np.asarray(eps, np.float64)
    lib().ora_project(n, _p(P.means), _p(P.coeffs), _p(P.scales), _p(P.quats),
                      _p(P.opacity), _p(P.amplitude), _p(P.delta_of(b)), _p(P.sh),
                      _p(pack_frame(scene, b)), _p(pack_sensor(scene)),
                      _p(pack_consts(scene)), _p(e), _p(out))
    return out


def render_frame(scene, b: int, splats=None, eps=EPS_NONE, bg=None):
    """(out (C,H,W), tfinal (H,W), ambig (H,W), ncontrib (H,W)) for frame b."""
    if splats is None:
        splats = project(scene, b, eps)
    C, H, W = n_channels(scene), scene.height, scene.width
    out = np.zeros((C, H, W))
    tf = np.zeros((H, W))
    amb = np.zeros((H, W), np.int32)
    nc = np.zeros((H, W), np.int32)
    bgb = _f64(scene.bg[b] if bg is None else bg)
    lib().ora_render_frame(scene.n, _p(splats), _p(pack_frame(scene, b)),
                           _p(pack_sensor(scene)), _p(pack_consts(scene)),
                           _p(bgb), _p(np.asarray(eps, np.float64)), _p(out),
                           _p(tf), _p(amb, _i32), _p(nc, _i32))
    return out, tf, amb, nc


def render_pixels(scene, b: int, pix: np.ndarray, splats=None, eps=EPS_NONE):
    """Samples at pixel list pix (k, 2) of frame b: (out (k,C), tfinal, ambig, ncontrib)."""
    if splats is None:
        splats = project(scene, b, eps)
    pix = np.ascontiguousarray(pix, np.int32)
    k, C = pix.shape[0], n_channels(scene)
    out = np.zeros((k, C))
    tf = np.zeros(k)
    amb = np.zeros(k, np.int32)
    nc = np.zeros(k, np.int32)
    lib().ora_render_pixels(scene.n, _p(splats), _p(pack_frame(scene, b)),
                            _p(pack_sensor(scene)), _p(pack_consts(scene)),
                            _p(_f64(scene.bg[b])), _p(np.asarray(eps, np.float64)),
                            k, _p(pix, _i32), _p(out), _p(tf), _p(amb, _i32),
                            _p(nc, _i32))
    return out, tf, amb, nc


def render_tiles(scene, b: int, tiles, splats=None, eps=EPS_F32, max_alt: int = 32,
                 alt_per_pixel: int = 8):
    """Whole tiles of frame b (tiles: (k, 2) of (tx, ty)) and every valid
    result of their ambiguous pixels.  Returns dict(pix (npix, 2) (x, y),
    out (npix, C), tfinal, ambig, alts {pixel index: (k, C) results, the
    nominal one first}, capped = pixels whose search hit max_alt)."""
    if splats is None:
        splats = project(scene, b, eps)
    tiles = np.ascontiguousarray(np.asarray(tiles, np.int32).reshape(-1, 2))
    k = scene.consts
    npix_max = len(tiles) * int(k.tile_w) * int(k.tile_h)
    C = n_channels(scene)
    out = np.zeros((npix_max, C))
    tf = np.zeros(npix_max)
    amb = np.zeros(npix_max, np.int32)
    pix = np.zeros((npix_max, 2), np.int32)
    cap = max(1, npix_max * alt_per_pixel)
    _i64 = ctypes.POINTER(ctypes.c_int64)
    while True:
        alt_out = np.zeros((cap, C))
        alt_pix = np.zeros(cap, np.int64)
        n_alt = np.zeros(1, np.int64)
        n_capped = np.zeros(1, np.int64)
        npix = lib().ora_render_tiles(scene.n, _p(splats), _p(pack_frame(scene, b)),
                                      _p(pack_sensor(scene)), _p(pack_consts(scene)),
                                      _p(_f64(scene.bg[b])), _p(np.asarray(eps, np.float64)),
                                      len(tiles), _p(tiles, _i32), _p(out), _p(tf),
                                      _p(amb, _i32), _p(pix, _i32), int(max_alt), cap,
                                      _p(alt_out), _p(alt_pix, _i64), _p(n_alt, _i64),
                                      _p(n_capped, _i64))
        if n_alt[0] <= cap:
            break
        cap = int(n_alt[0])
    alts = {}
    m = int(n_alt[0])
    for i in range(m):
        alts.setdefault(int(alt_pix[i]), []).append(alt_out[i])
    alts = {p_: np.stack(v) for p_, v in alts.items()}
    return dict(pix=pix[:npix], out=out[:npix], tfinal=tf[:npix], ambig=amb[:npix],
                alts=alts, capped=int(n_capped[0]))


def pixel_steps(scene, b: int, x: int, y: int, splats=None, max_steps: int = 100000):
    """Instrumented pixel (x, y) of frame b: (alpha_k, T_k) of the composited
    Gaussians front to back (T_k one-way, before Gaussian k) and T_N."""
    if splats is None:
        splats = project(scene, b)
    alpha = np.zeros(max_steps)
    trans = np.zeros(max_steps)
    tf = np.zeros(1)
    k = lib().ora_pixel_steps(scene.n, _p(splats), _p(pack_sensor(scene)),
                              _p(pack_consts(scene)), _p(np.asarray(EPS_NONE, np.float64)),
                              int(x), int(y), max_steps, _p(alpha), _p(trans), _p(tf))
    k = min(k, max_steps)
    return alpha[:k], trans[:k], float(tf[0])


def render(scene, eps=EPS_NONE, params: Params = None):
    """All frames: out (B,C,H,W), tfinal (B,H,W), ambig (B,H,W), ncontrib."""
    outs, tfs, ambs, ncs = [], [], [], []
    for b in range(scene.frames):
        sp = project(scene, b, eps, params)
        o, t, a, c = render_frame(scene, b, sp, eps)
        outs.append(o), tfs.append(t), ambs.append(a), ncs.append(c)
    return np.stack(outs), np.stack(tfs), np.stack(ambs), np.stack(ncs)


def backward(scene, dout: np.ndarray, params: Params = None, want_2d=False):
    """Analytic FP64 gradient of L = sum(dout * render(scene)).

    Returns a dict with means (N,3), coeffs (N,3,3), scales (N,3), quats (N,4),
    opacity (N,), amplitude (N,), delta (B,N,3), bg (B,C), sh (N, n_sh) when
    the scene has SH reflectivity and, when want_2d,
    g2d (B, N, 7+2F+1) -- gradients w.r.t. (u, v, conic a, b, c, opacity,
    features, distance)."""
    P = params or Params(scene)
    n, B = scene.n, scene.frames
    nf = 2 * len(scene.sensor.freqs_hz) + 1
    C = n_channels(scene)
    grads = np.zeros((n, NPARAM))
    gdelta = np.zeros((B, n, 3))
    gbg = np.zeros((B, C))
    g2ds = []
    se, co = pack_sensor(scene), pack_consts(scene)
    for b in range(B):
        sp = project(scene, b, EPS_NONE, P)
        fr = pack_frame(scene, b)
        g2d = np.zeros((n, 7 + nf))
        db = np.ascontiguousarray(dout[b], np.float64)
        lib().ora_backward_2d(n, _p(sp), _p(fr), _p(se), _p(co),
                              _p(_f64(scene.bg[b])), _p(db), _p(g2d), _p(gbg[b]))
        gb = np.zeros((n, NPARAM))
        lib().ora_backward_params(n, _p(P.means), _p(P.coeffs), _p(P.scales),
                                  _p(P.quats), _p(P.opacity), _p(P.amplitude),
                                  _p(P.delta_of(b)), _p(P.sh), _p(fr), _p(se), _p(co),
                                  _p(sp), _p(g2d), _p(gb))
        grads += gb
        gdelta[b] = gb[:, 21:24]
        if want_2d:
            g2ds.append(g2d)
    out = dict(means=grads[:, 0:3], coeffs=grads[:, 3:12].reshape(n, 3, 3),
               scales=grads[:, 12:15], quats=grads[:, 15:19],
               opacity=grads[:, 19], amplitude=grads[:, 20], delta=gdelta,
               bg=gbg)
    if n_sh(scene):
        out["sh"] = grads[:, 24:24 + n_sh(scene)].copy()
    if want_2d:
        out["g2d"] = np.stack(g2ds)
    return out


def bin_f32(u, v, radius, z, width, height, tile_w, tile_h, capacity=None):
    """Bit-exact binning contract: (keys u64[M], values u32[M],
    ranges u32[B*tiles, 2]) from float32 footprints shaped (B, N)."""
    u = np.ascontiguousarray(u, np.float32)
    v = np.ascontiguousarray(v, np.float32)
    z = np.ascontiguousarray(z, np.float32)
    radius = np.ascontiguousarray(radius, np.int32)
    B, n = u.shape
    tiles = ((width + tile_w - 1) // tile_w) * ((height + tile_h - 1) // tile_h)
    if capacity is None:
        capacity = 0
        r = radius.astype(np.int64)
        capacity = int(np.sum(((2 * r + tile_w) // tile_w + 2) * ((2 * r + tile_h) // tile_h + 2)))
    keys = np.zeros(max(capacity, 1), np.uint64)
    vals = np.zeros(max(capacity, 1), np.uint32)
    ranges = np.zeros((B * tiles, 2), np.uint32)
    m = lib().ora_bin_f32(n, B, _p(u, _f32), _p(v, _f32), _p(radius, _i32),
                          _p(z, _f32), width, height, tile_w, tile_h, capacity,
                          _p(keys, _u64), _p(vals, _u32), _p(ranges, _u32))
    if m < 0:
        raise RuntimeError("oracle binning capacity exceeded")
    return keys[:m].copy(), vals[:m].copy(), ranges
