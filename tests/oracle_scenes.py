"""Hand-built tiny scenes for the oracle pin tests (inputs only)."""
import math

import numpy as np

from paper_2505_05356_gb300 import scenes

C_LIGHT = 299792458.0


def tiny_scene(positions, scales, quats=None, opacity=None, amplitude=None,
               width=64, height=64, freqs=(30e6,), offsets=None, bg=None,
               coeffs=None, times=(0.0,), world_to_cam=None, consts=None,
               source_intensity=1.0, delta=None, sh=None, frame_phase=None,
               interp_times=None):
    """Scene with the given Gaussians (float64 values kept exactly)."""
    positions = np.asarray(positions, np.float64).reshape(-1, 3)
    n = positions.shape[0]
    scales = np.broadcast_to(np.asarray(scales, np.float64), (n, 3)).copy()
    if quats is None:
        quats = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    quats = np.asarray(quats, np.float64).reshape(n, 4)
    opacity = np.full(n, 0.5) if opacity is None else np.asarray(opacity, np.float64)
    amplitude = np.full(n, 1.0) if amplitude is None else np.asarray(amplitude, np.float64)
    if offsets is None:
        offsets = [0.0, math.pi / 2, math.pi, 3 * math.pi / 2]
    sensor = scenes.Sensor(list(freqs), list(offsets), source_intensity)
    cam = scenes.pinhole(width, height)
    if world_to_cam is not None:
        cam.world_to_cam = np.asarray(world_to_cam, np.float64)
    frames = len(times)
    consts = consts or scenes.Consts()
    C = sensor.n_channels + (2 * len(freqs) if consts.phasor else 0) + (1 if consts.depth else 0)
    if bg is None:
        bg = np.zeros((frames, C))
    bg = np.broadcast_to(np.asarray(bg, np.float64), (frames, C)).copy()
    return scenes.Scene(positions, coeffs, scales, quats, opacity, amplitude,
                        np.asarray(times, np.float64), [cam] * frames, delta,
                        sensor, consts, bg,
                        None if sh is None else np.asarray(sh, np.float64).reshape(n, -1),
                        None if frame_phase is None else np.asarray(frame_phase, np.float64),
                        None if interp_times is None else
                        np.asarray(interp_times, np.float64).reshape(frames, 2))


def at_pixel(cam, px, py, z):
    """World point at depth z projecting exactly onto position (px, py)."""
    return [(px - cam.cx) * z / cam.fx, (py - cam.cy) * z / cam.fy, z]
