"""Seeded synthetic scenes shaped like the paper's C-ToF workloads.

This module only DRAWS inputs (random Gaussian parameters, cameras, times,
backgrounds); it holds none of the method's arithmetic.  Both the CUDA path's
tests and the FP64 oracle take their inputs from here.  Every array is drawn
in single precision and kept as float32, so the single-precision CUDA path and
the double-precision oracle see exactly the same numbers (the oracle widens
them losslessly).

Scene shapes (the paper's datasets are not available; these stand in for
their shape: a static monocular camera, fast lateral/axial motion, depths
within about one unambiguous range, raw quartets; Sec. 5 "Datasets"):

* ``static_1k``   -- 1,000 static Gaussians, 64x64, 30 MHz, 4 offsets.
* ``dynamic_100k`` -- 100,000 Gaussians on cubic trajectories, 640x480.
* ``batch_300k``  -- 300,000 dynamic Gaussians, 640x480, 16 timesteps t=b/15,
  per-frame visible fraction U[0.3, 1] (the rest displaced 10 m sideways
  for that frame through the per-frame displacement input).
* ``twofreq_500k`` -- 500,000 dynamic Gaussians, 640x576, 30 and 80 MHz
  (phase wrapping), depths 0.5-6 m, 8 timesteps.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

F32 = np.float32


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    world_to_cam: np.ndarray  # (3, 4) float32, [R | t], R orthonormal
    near: float = 0.2


@dataclasses.dataclass
class Sensor:
    freqs_hz: List[float]
    offsets_rad: List[float]
    source_intensity: float = 1.0

    @property
    def n_channels(self) -> int:
        return len(self.freqs_hz) * len(self.offsets_rad) + 1


@dataclasses.dataclass
class Consts:
    dilation: float = 0.3
    alpha_max: float = 0.99
    alpha_min: float = 1.0 / 255.0
    t_min: float = 1e-4
    guard: float = 1.3
    sigma_cut: float = 3.0
    tile_w: int = 16
    tile_h: int = 16
    phasor: bool = False  # extra Eq. 3 phasor channels (Re, Im per frequency)
    depth: bool = False   # extra Eq. 5 mean-depth channel

    def rounded(self) -> "Consts":
        """The same constants rounded to float32 (what a single-precision
        implementation actually uses)."""
        r = lambda v: float(np.float32(v))
        return Consts(r(self.dilation), r(self.alpha_max), r(self.alpha_min),
                      r(self.t_min), r(self.guard), r(self.sigma_cut),
                      self.tile_w, self.tile_h, self.phasor, self.depth)


@dataclasses.dataclass
class Scene:
    means: np.ndarray       # (N, 3)
    coeffs: Optional[np.ndarray]  # (N, 3, 3): c1, c2, c3 (each xyz)
    scales: np.ndarray      # (N, 3) linear scales
    quats: np.ndarray       # (N, 4) w, x, y, z (unnormalised)
    opacity: np.ndarray     # (N,) in (0, 1)
    amplitude: np.ndarray   # (N,) reflectivity r_k
    times: np.ndarray       # (B,)
    cameras: List[Camera]   # B cameras
    delta: Optional[np.ndarray]  # (B, N, 3) per-frame displacement or None
    sensor: Sensor
    consts: Consts
    bg: np.ndarray          # (B, C) background per channel
    sh: Optional[np.ndarray] = None  # (N, n_sh) SH reflectivity, n_sh in 1,4,9,16
    frame_phase: Optional[np.ndarray] = None   # (B,) rad added to the offsets
    interp_times: Optional[np.ndarray] = None  # (B, 2) Eq. 7 bracketing timesteps

    @property
    def n_sh(self) -> int:
        return 0 if self.sh is None else int(self.sh.shape[1])

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def n_channels(self) -> int:
        """Raw samples + ambient (+ phasor Re, Im per frequency) (+ depth)."""
        F = len(self.sensor.freqs_hz)
        return (self.sensor.n_channels + (2 * F if self.consts.phasor else 0) +
                (1 if self.consts.depth else 0))

    @property
    def frames(self) -> int:
        return len(self.cameras)

    @property
    def width(self) -> int:
        return self.cameras[0].width

    @property
    def height(self) -> int:
        return self.cameras[0].height


def pinhole(width: int, height: int, fov_x_deg: float = 60.0,
            near: float = 0.2) -> Camera:
    """Camera at the origin looking down +z, square pixels, principal point
    at the image centre (fx from the horizontal field of view)."""
    fx = float(F32(width / (2.0 * math.tan(math.radians(fov_x_deg) / 2.0))))
    rt = np.zeros((3, 4), F32)
    rt[:3, :3] = np.eye(3, dtype=F32)
    return Camera(width, height, fx, fx, width / 2.0, height / 2.0, rt, near)


def _unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(F32)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _rotation_xyz(rx, ry, rz) -> np.ndarray:
    """Rotation about x, then y, then z (angles in degrees)."""
    a, b, c = (math.radians(v) for v in (rx, ry, rz))
    Rx = np.array([[1, 0, 0], [0, math.cos(a), -math.sin(a)], [0, math.sin(a), math.cos(a)]])
    Ry = np.array([[math.cos(b), 0, math.sin(b)], [0, 1, 0], [-math.sin(b), 0, math.cos(b)]])
    Rz = np.array([[math.cos(c), -math.sin(c), 0], [math.sin(c), math.cos(c), 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def random_gaussians(rng, n, cam: Camera, z_range=(1.0, 3.0), box=False,
                     log_scale=(-3.5, 0.3), coeff_std=0.0):
    """Random Gaussians: depth uniform in z_range, lateral position uniform
    inside the camera frustum at that depth (or in a 1 m box when box=True)."""
    z = rng.uniform(z_range[0], z_range[1], n)
    if box:
        x = rng.uniform(-0.5, 0.5, n)
        y = rng.uniform(-0.5, 0.5, n)
    else:
        hx = (cam.width / 2.0) / cam.fx
        hy = (cam.height / 2.0) / cam.fy
        x = rng.uniform(-1.0, 1.0, n) * hx * z
        y = rng.uniform(-1.0, 1.0, n) * hy * z
    means = np.stack([x, y, z], 1).astype(F32)
    scales = np.exp(rng.normal(log_scale[0], log_scale[1], (n, 3))).astype(F32)
    quats = _unit_quats(rng, n)
    opacity = _sigmoid(rng.standard_normal(n)).astype(F32)
    amplitude = rng.uniform(0.1, 1.0, n).astype(F32)
    coeffs = None
    if coeff_std > 0:
        coeffs = rng.normal(0.0, coeff_std, (n, 3, 3)).astype(F32)
    return means, coeffs, scales, quats, opacity, amplitude


def make_scene(name: str, seed: int = 0, **over) -> Scene:
    """Build one of the named synthetic workloads (see module docstring).

    Overrides: n, width, height, frames, freqs_hz, offsets_rad, tile, bg
    ('zero' | 'random'), z_range, coeff_std, visible_min, consts, phasor,
    depth, sh_degree (0..3: view-dependent reflectivity from (degree+1)^2 SH
    coefficients; the DC term reproduces the scalar amplitude draw, the others
    are N(0, sh_std) with sh_std 0.03 by default), pose ((rx, ry, rz) degrees
    of an x-then-y-then-z rotation, optical centre (cx, cy, cz)): a moved
    camera, with the Gaussians drawn in its frustum and stored in world
    coordinates.  async_capture=True: asynchronous raw capture (Sec. 3), one
    raw sample per frame (P = 1, sensor offset 0) with frame b at tick b
    (t_b = b / (B - 1)) sampling phase offset (pi/2) (b mod 4); the first frame
    of each quartet is an integer timestep and the others interpolate the
    positions linearly between it and the next quartet's first frame (Eq. 7).
    """
    rng = np.random.default_rng(seed)
    if name == "static_1k":
        d = dict(n=1000, width=64, height=64, frames=1, freqs_hz=[30e6],
                 z_range=(1.0, 3.0), coeff_std=0.0, box=True, visible_min=1.0)
    elif name == "dynamic_100k":
        d = dict(n=100_000, width=640, height=480, frames=1, freqs_hz=[30e6],
                 z_range=(1.0, 3.0), coeff_std=0.05, box=False, visible_min=1.0)
    elif name == "batch_300k":
        d = dict(n=300_000, width=640, height=480, frames=16, freqs_hz=[30e6],
                 z_range=(1.0, 3.0), coeff_std=0.05, box=False, visible_min=0.3)
    elif name == "twofreq_500k":
        d = dict(n=500_000, width=640, height=576, frames=8,
                 freqs_hz=[30e6, 80e6], z_range=(0.5, 6.0), coeff_std=0.05,
                 box=False, visible_min=0.3)
    else:
        raise ValueError("unknown scene %r" % name)
    d.update(dict(offsets_rad=[0.0, math.pi / 2, math.pi, 3 * math.pi / 2],
                  tile=(16, 16), bg="random", log_scale=(-3.5, 0.3)))
    d.update(over)
    if d.get("async_capture"):
        d["offsets_rad"] = [0.0]

    cam = pinhole(d["width"], d["height"])
    means, coeffs, scales, quats, opacity, amplitude = random_gaussians(
        rng, d["n"], cam, d["z_range"], d["box"], d["log_scale"], d["coeff_std"])
    if d.get("pose") is not None:
        R = _rotation_xyz(*d["pose"][0])
        centre = np.asarray(d["pose"][1], np.float64)
        rt = np.concatenate([R, (-R @ centre)[:, None]], 1).astype(F32)
        cam.world_to_cam = rt
        R32 = rt[:, :3].astype(np.float64)
        means = (means.astype(np.float64) @ R32 + centre).astype(F32)
    frames = d["frames"]
    times = (np.arange(frames) / max(frames - 1, 1)).astype(F32)
    if frames == 1 and d["coeff_std"] > 0:
        times = np.array([rng.uniform(0.0, 1.0)], F32)
    delta = None
    if d["visible_min"] < 1.0:
        delta = np.zeros((frames, d["n"], 3), F32)
        for b in range(frames):
            v = rng.uniform(d["visible_min"], 1.0)
            hide = rng.random(d["n"]) >= v
            delta[b, hide, 0] = 10.0
    sensor = Sensor([float(F32(f)) for f in d["freqs_hz"]],
                    [float(F32(o)) for o in d["offsets_rad"]], 1.0)
    consts = d.get("consts") or Consts(tile_w=d["tile"][0], tile_h=d["tile"][1],
                                       phasor=d.get("phasor", False),
                                       depth=d.get("depth", False))
    consts = consts.rounded()
    C = sensor.n_channels + (2 * len(sensor.freqs_hz) if consts.phasor else 0) + \
        (1 if consts.depth else 0)
    if d["bg"] == "random":
        bg = rng.uniform(-1.0, 1.0, (frames, C)).astype(F32)
    else:
        bg = np.zeros((frames, C), F32)
    sh = None
    deg = d.get("sh_degree")
    if deg is not None:
        k = (int(deg) + 1) ** 2
        sh = rng.normal(0.0, d.get("sh_std", 0.03), (d["n"], k))
        # DC basis value 1 / (2 sqrt(pi)): r = 0.5 + sh_0 Y_0 + ... = amplitude + ...
        sh[:, 0] = (amplitude - 0.5) * (2.0 * math.sqrt(math.pi))
        sh = sh.astype(F32)
    phase = interp = None
    if d.get("async_capture"):
        tick = 1.0 / max(frames - 1, 1)
        phase = np.array([(math.pi / 2) * (b % 4) for b in range(frames)], F32)
        t0 = np.array([4 * (b // 4) * tick for b in range(frames)])
        interp = np.stack([t0, t0 + 4 * tick], 1).astype(F32)
    return Scene(means, coeffs, scales, quats, opacity, amplitude, times,
                 [cam] * frames, delta, sensor, consts, bg, sh, phase, interp)


def random_dout(scene: Scene, seed: int = 1, density: float = 1.0) -> np.ndarray:
    """A seeded loss gradient dL/d(out), shape (B, C, H, W), float32.
    density < 1 keeps only that fraction of pixels (the rest exactly 0)."""
    rng = np.random.default_rng(seed)
    B, C, H, W = scene.frames, scene.n_channels, scene.height, scene.width
    g = rng.standard_normal((B, C, H, W)).astype(F32)
    if density < 1.0:
        keep = rng.random((B, 1, H, W)) < density
        g = g * keep
    return g


def sample_pixels(scene: Scene, k: int, seed: int = 2) -> np.ndarray:
    """k distinct pixel positions (x, y) per frame, int32, shape (B, k, 2)."""
    rng = np.random.default_rng(seed)
    out = np.zeros((scene.frames, k, 2), np.int32)
    for b in range(scene.frames):
        idx = rng.choice(scene.width * scene.height, size=k, replace=False)
        out[b, :, 0] = idx % scene.width
        out[b, :, 1] = idx // scene.width
    return out


def sample_tiles(scene: Scene, k: int, seed: int = 2) -> np.ndarray:
    """k distinct tiles (tx, ty) of the scene's tile grid per frame, int32,
    shape (B, k, 2)."""
    rng = np.random.default_rng(seed)
    tw, th = scene.consts.tile_w, scene.consts.tile_h
    nx, ny = -(-scene.width // tw), -(-scene.height // th)
    out = np.zeros((scene.frames, k, 2), np.int32)
    for b in range(scene.frames):
        idx = rng.choice(nx * ny, size=k, replace=False)
        out[b, :, 0] = idx % nx
        out[b, :, 1] = idx // nx
    return out


def make_fit_scenes(seed: int = 4, n_backdrop: int = 270_000, n_rod: int = 30_000,
                    n_init: int = 300_000, frames: int = 60, width: int = 640,
                    height: int = 480):
    """Ground truth and initial guess of the optimisation-loop workload.

    Ground truth: a static backdrop (a wall at z = 5 m and a 1 m box around
    z = 3.5 m, n_backdrop surface Gaussians) and an elongated object (a 0.8 m
    rod of n_rod Gaussians, scales elongated along it) swinging about a pivot
    in the image plane, theta(t) = A sin(pi t) with a 2 m/s peak tip speed,
    seen in `frames` raw frames at t = b / (frames - 1) (the swing enters
    through the per-frame displacement).  Initial guess (Sec. 4,
    "Initialization"): n_init Gaussians uniform in the frustum between 1 and
    6 m, reflectivity 0.1, static (zero trajectory coefficients).
    Returns (gt, init) Scenes sharing cameras, times and sensor.
    """
    rng = np.random.default_rng(seed)
    cam = pinhole(width, height)
    hx, hy = (width / 2.0) / cam.fx, (height / 2.0) / cam.fy
    # backdrop: 70 % on the wall, 30 % on the box faces
    n_wall = int(0.7 * n_backdrop)
    n_box = n_backdrop - n_wall
    wall = np.stack([rng.uniform(-1, 1, n_wall) * hx * 5.0, rng.uniform(-1, 1, n_wall) * hy * 5.0,
                     np.full(n_wall, 5.0) + rng.normal(0, 0.005, n_wall)], 1)
    face = rng.integers(0, 6, n_box)
    uv = rng.uniform(-0.5, 0.5, (n_box, 2))
    box = np.zeros((n_box, 3))
    ax = face // 2
    sgn = np.where(face % 2 == 0, -0.5, 0.5)
    for a in range(3):
        on = ax == a
        others = [k for k in range(3) if k != a]
        box[on, a] = sgn[on]
        box[on, others[0]] = uv[on, 0]
        box[on, others[1]] = uv[on, 1]
    box += np.array([0.8, 0.4, 3.5])
    # rod along +x from the pivot at rest, swinging in the x-y plane
    pivot = np.array([-0.9, -0.3, 2.5])
    s_along = rng.uniform(0.0, 0.8, n_rod)
    rod = pivot + np.stack([s_along, rng.normal(0, 0.01, n_rod), rng.normal(0, 0.01, n_rod)], 1)
    means = np.concatenate([wall, box, rod]).astype(F32)
    n = means.shape[0]
    scales = np.empty((n, 3))
    scales[:n_backdrop] = np.exp(rng.normal(-4.2, 0.2, (n_backdrop, 3)))
    scales[n_backdrop:] = np.stack([np.exp(rng.normal(-3.9, 0.1, n_rod)),
                                    np.exp(rng.normal(-5.0, 0.1, n_rod)),
                                    np.exp(rng.normal(-5.0, 0.1, n_rod))], 1)
    quats = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    quats[:n_backdrop] = _unit_quats(rng, n_backdrop)
    opacity = np.concatenate([rng.uniform(0.6, 0.99, n_backdrop), np.full(n_rod, 0.95)])
    amplitude = np.concatenate([rng.uniform(0.3, 0.9, n_backdrop), np.full(n_rod, 0.8)])
    times = (np.arange(frames) / max(frames - 1, 1)).astype(F32)
    A = 2.0 / (0.8 * math.pi)  # peak angular speed A pi, tip speed 0.8 A pi = 2 m/s
    delta = np.zeros((frames, n, 3), F32)
    rel = means[n_backdrop:].astype(np.float64) - pivot
    for b, t in enumerate(times):
        th = A * math.sin(math.pi * float(t))
        c, s_ = math.cos(th), math.sin(th)
        rot = np.stack([c * rel[:, 0] - s_ * rel[:, 1], s_ * rel[:, 0] + c * rel[:, 1],
                        rel[:, 2]], 1)
        delta[b, n_backdrop:] = (rot - rel).astype(F32)
    sensor = Sensor([float(F32(30e6))], [float(F32(o)) for o in
                                         (0.0, math.pi / 2, math.pi, 3 * math.pi / 2)], 1.0)
    consts = Consts().rounded()
    bg = np.zeros((frames, sensor.n_channels), F32)
    gt = Scene(means, None, scales.astype(F32), quats.astype(F32), opacity.astype(F32),
               amplitude.astype(F32), times, [cam] * frames, delta, sensor, consts, bg)
    m0, _, s0, q0, o0, _ = random_gaussians(rng, n_init, cam, (1.0, 6.0))
    init = Scene(m0, np.zeros((n_init, 3, 3), F32), s0, q0, o0, np.full(n_init, 0.1, F32),
                 times, [cam] * frames, None, sensor, consts, bg.copy())
    return gt, init


def init_mlp_params(seed: int = 0, head_std: float = 1e-5, width: int = 256, depth: int = 8,
                    in_pad: int = 128, in_used: int = 84) -> np.ndarray:
    """Packed float32 parameters of the deformation MLP (layout in
    paper_2505_05356_gb300/mlp.py) drawn as in Sec. 4 ("MLP"): zero biases,
    Xavier-normal hidden weights (std sqrt(2 / (fan_in + fan_out)), fan_in the
    84 used inputs for the first layer, whose padding columns are 0), and the
    head drawn from N(0, head_std) (1e-5 in the paper)."""
    rng = np.random.default_rng(seed)
    parts = []
    for li in range(depth):
        fan_in = in_used if li == 0 else width
        k = in_pad if li == 0 else width
        W = np.zeros((width, k))
        W[:, :fan_in] = rng.normal(0.0, math.sqrt(2.0 / (fan_in + width)), (width, fan_in))
        parts += [W.reshape(-1), np.zeros(width)]
    parts += [rng.normal(0.0, head_std, 3 * width), np.zeros(3)]
    return np.concatenate(parts).astype(F32)
