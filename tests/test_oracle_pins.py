"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms (Sec. 2 quad model, Eq. 1 depth, Eq. 4 with squared transmittance),
special cases that reduce to a library routine (scipy rotations, numpy
linear algebra), brute force on tiny inputs, and central finite differences
of its own forward for its analytic gradient (Eq. S3 + projection chain).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as ora
from tests.oracle_scenes import C_LIGHT, at_pixel, tiny_scene

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                     "closed_forms.json")))
SP = ora.SP


def _render_px(scene, px, py, b=0):
    out, tf, amb, nc = ora.render_pixels(scene, b, np.array([[px, py]], np.int32))
    return out[0], tf[0], nc[0]


# --------------------------------------------------------------------------
# image formation (Sec. 2, Eq. 1, Eq. 4)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("d,f", [(2.0, 30e6), (1.3, 30e6), (2.0, 80e6), (6.0, 30e6)])
def test_single_opaque_gaussian_quads_and_depth(d, f):
    """One opaque Gaussian centred on a pixel: alpha clamps at 0.99, so
    Q_j = 0.99 (s r / d^2) sin(psi + phi_j) + 0.01 bg_j with psi = 4 pi d f/c
    (Eq. 4 with one term, T_N = 0.01), and Eq. 1 recovers d mod d_u."""
    sc0 = tiny_scene([[0, 0, 1]], 0.05)
    cam = sc0.cameras[0]
    # put the Gaussian at Euclidean distance d, projecting onto pixel (40, 21)
    p = np.array(at_pixel(cam, 40.5, 21.5, 1.0))
    pos = p / np.linalg.norm(p) * d
    bg = np.array([0.3, 0.3, 0.3, 0.3, -0.5])  # one bias B for the quartet
    r, s = 0.6, 1.7
    sc = tiny_scene([pos], 0.02 * d, opacity=[0.9999], amplitude=[r], freqs=(f,),
                    bg=bg, source_intensity=s)
    q, T, k = _render_px(sc, 40, 21)
    assert k == 1 and abs(T - 0.01) < 1e-12
    psi = 4 * math.pi * d * f / C_LIGHT
    A = s * r / d ** 2
    phis = GOLDEN["phase_offsets_rad"]["value"]
    for j, phi in enumerate(phis):
        assert q[j] == pytest.approx(0.99 * A * math.sin(psi + phi) + 0.01 * bg[j], abs=1e-12)
    # ambient channel: falloff-weighted amplitude plus background
    assert q[4] == pytest.approx(0.99 * A + 0.01 * bg[4], abs=1e-12)
    # Eq. 1: the quad differences cancel a common background bias exactly
    psi_rec = math.atan2(q[0] - q[2], q[1] - q[3]) % (2 * math.pi)
    d_u = C_LIGHT / (2 * f)
    d_rec = C_LIGHT * psi_rec / (4 * math.pi * f)
    assert d_rec == pytest.approx(d % d_u, abs=1e-9)
    # amplitude relation of Sec. 2: A = 1/2 sqrt((Q0-Qpi)^2 + (Qpi/2-Q3pi/2)^2)
    amp = 0.5 * math.hypot(q[0] - q[2], q[1] - q[3])
    assert amp == pytest.approx(0.99 * A, rel=1e-12)


def test_golden_phase_and_range():
    """Golden closed forms of Sec. 2: psi at 2 m, wrapping at 80 MHz, d_u."""
    for case in GOLDEN["unambiguous_range"]["cases"]:
        assert C_LIGHT / (2 * case["f_hz"]) == pytest.approx(case["d_u_m"], rel=1e-15)
    c30, c80 = GOLDEN["phase_of_depth"]["cases"]
    p = np.array(at_pixel(tiny_scene([[0, 0, 1]], 0.1).cameras[0], 32.5, 32.5, 1.0))
    pos = p / np.linalg.norm(p) * c30["d_m"]  # Euclidean distance 2 m
    sc = tiny_scene([pos], 0.04, opacity=[0.9999], freqs=(c30["f_hz"], c80["f_hz"]))
    q, T, _ = _render_px(sc, 32, 32)
    psi30 = math.atan2(q[0] - q[2], q[1] - q[3]) % (2 * math.pi)
    psi80 = math.atan2(q[4] - q[6], q[5] - q[7]) % (2 * math.pi)
    assert psi30 == pytest.approx(c30["psi_rad"], abs=1e-10)
    assert psi80 == pytest.approx(c80["psi_wrapped_rad"], abs=1e-10)
    d80 = C_LIGHT * psi80 / (4 * math.pi * c80["f_hz"])
    assert d80 == pytest.approx(c80["d_tof_m"], abs=1e-10)


def test_phase_wrap_equivalence():
    """A Gaussian at d and one at d + d_u (falloff compensated through the
    amplitude) give identical raw samples (Sec. 2 phase wrapping)."""
    f = 80e6
    d_u = C_LIGHT / (2 * f)
    cam = tiny_scene([[0, 0, 1]], 0.1).cameras[0]
    outs = []
    for d in (1.1, 1.1 + d_u):
        p = np.array(at_pixel(cam, 32.5, 32.5, 1.0))
        pos = p / np.linalg.norm(p) * d
        sc = tiny_scene([pos], 0.02 * d, opacity=[0.9999],
                        amplitude=[(d / 1.1) ** 2], freqs=(f,))
        outs.append(_render_px(sc, 32, 32)[0])
    np.testing.assert_allclose(outs[0], outs[1], rtol=0, atol=1e-12)


def test_two_gaussians_squared_transmittance():
    """Two Gaussians on one pixel: the second is weighted by (1 - a1)^2
    (round trip, Eq. 4) and the background by the one-way T_N = (1-a1)(1-a2)."""
    cam = tiny_scene([[0, 0, 1]], 0.1).cameras[0]
    pa = at_pixel(cam, 20.5, 30.5, 1.2)
    pb = at_pixel(cam, 20.5, 30.5, 2.5)
    o1, o2 = 0.4, 0.7
    bg = np.array([0.5, 0.25, -0.75, 0.1, 0.3])
    sc = tiny_scene([pb, pa], 0.03, opacity=[o2, o1], amplitude=[0.8, 0.5], bg=bg)
    q, T, k = _render_px(sc, 20, 30)
    assert k == 2
    d1, d2 = np.linalg.norm(pa), np.linalg.norm(pb)
    A1, A2 = 0.5 / d1 ** 2, 0.8 / d2 ** 2
    ps1, ps2 = (4 * math.pi * d * 30e6 / C_LIGHT for d in (d1, d2))
    assert T == pytest.approx((1 - o1) * (1 - o2), abs=1e-14)
    for j, phi in enumerate(GOLDEN["phase_offsets_rad"]["value"]):
        want = (o1 * A1 * math.sin(ps1 + phi) + o2 * (1 - o1) ** 2 * A2 * math.sin(ps2 + phi)
                + bg[j] * (1 - o1) * (1 - o2))
        assert q[j] == pytest.approx(want, abs=1e-13)
    assert q[4] == pytest.approx(o1 * A1 + o2 * (1 - o1) ** 2 * A2 + bg[4] * T, abs=1e-13)


def test_telescoping_coincident_gaussians():
    """N coincident Gaussians with equal alpha: sum alpha T_k^2 is the golden
    geometric series and T_N = (1 - alpha)^N (ties broken by index)."""
    case = GOLDEN["telescoping"]["cases"][0]
    cam = tiny_scene([[0, 0, 1]], 0.1).cameras[0]
    p = at_pixel(cam, 10.5, 50.5, 2.0)
    d = float(np.linalg.norm(p))
    n = case["N"]
    sc = tiny_scene([p] * n, 0.05, opacity=[case["alpha"]] * n,
                    amplitude=[d * d] * n)  # A = s r / d^2 = 1
    q, T, k = _render_px(sc, 10, 50)
    assert k == n
    assert T == pytest.approx(case["T_final"], abs=1e-15)
    assert q[4] == pytest.approx(case["sum_weights"], abs=1e-14)
    a = case["alpha"]
    assert case["sum_weights"] == pytest.approx(a * (1 - (1 - a) ** (2 * n)) / (1 - (1 - a) ** 2))


def test_empty_scene_returns_background():
    """No visible Gaussian: Q = bg exactly, T_N = 1, zero gradients."""
    bg = np.array([0.25, -0.5, 0.125, 1.0, -2.0])
    sc = tiny_scene([[0, 0, -1.0], [0.1, 0, 0.1]], 0.05, bg=bg)  # behind / before near
    out, tf, amb, nc = ora.render(sc)
    assert np.all(tf == 1.0) and np.all(nc == 0)
    for c in range(5):
        assert np.all(out[0, c] == bg[c])
    g = ora.backward(sc, np.ones_like(out))
    for key in ("means", "scales", "quats", "opacity", "amplitude"):
        assert np.all(g[key] == 0.0)
    assert np.allclose(g["bg"][0], 64 * 64)  # dL/dbg = sum over pixels of T_N


def test_offset_cancellation_and_linearity():
    """Q_0 + Q_pi = (bg_0 + bg_pi) T_N (sinusoids cancel), and samples at an
    arbitrary offset are the same linear combination of the sine/cosine
    sums: Q(phi) - bg T = cos(phi)(Q_0 - bg_0 T) + sin(phi)(Q_pi/2 - bg T)."""
    from paper_2505_05356_gb300 import scenes
    sc = scenes.make_scene("static_1k", 3, n=300, width=48, height=40)
    sc.sensor.offsets_rad = list(GOLDEN["phase_offsets_rad"]["value"])  # exact
    out, tf, _, _ = ora.render(sc)
    bg = sc.bg[0]
    np.testing.assert_allclose(out[0, 0] + out[0, 2], (bg[0] + bg[2]) * tf[0], atol=1e-12)
    np.testing.assert_allclose(out[0, 1] + out[0, 3], (bg[1] + bg[3]) * tf[0], atol=1e-12)
    sc2 = scenes.make_scene("static_1k", 3, n=300, width=48, height=40,
                            offsets_rad=[0.3, 2.0, -1.1])
    sc2.bg = np.zeros((1, 4))
    out2, tf2, _, _ = ora.render(sc2)
    S = out[0, 0] - bg[0] * tf[0]
    Cc = out[0, 1] - bg[1] * tf[0]
    for j, phi in enumerate(sc2.sensor.offsets_rad):
        np.testing.assert_allclose(out2[0, j], math.cos(phi) * S + math.sin(phi) * Cc, atol=1e-12)


def test_zero_frequency_reduces_to_squared_3dgs():
    """f = 0: the sine sum vanishes and the cosine sum equals the ambient
    (falloff-weighted) sum, i.e. 3DGS Eq. 2 with T^2 and colour A_k."""
    from paper_2505_05356_gb300 import scenes
    sc = scenes.make_scene("static_1k", 4, n=200, width=32, height=32, freqs_hz=[0.0])
    sc.bg[:] = 0
    out, tf, _, _ = ora.render(sc)
    np.testing.assert_allclose(out[0, 0], 0.0, atol=1e-14)  # sin(0 + 0)
    np.testing.assert_allclose(out[0, 1], out[0, 4], atol=1e-14)  # offset pi/2


def test_alpha_floor_and_early_stop():
    """alpha < 1/255 is skipped; the Gaussian that would take T below 1e-4
    stops the walk without being composited (3DGS rules the paper keeps)."""
    cam = tiny_scene([[0, 0, 1]], 0.1).cameras[0]
    ps = [at_pixel(cam, 30.5, 30.5, z) for z in (1.0, 1.5, 2.0, 2.5)]
    # first: alpha 0.003 (< 1/255) -> skipped; then 0.98, 0.98, 0.98
    sc = tiny_scene(ps, 0.03, opacity=[0.003, 0.98, 0.98, 0.98],
                    amplitude=[1, 1, 1, 1])
    q, T, k = _render_px(sc, 30, 30)
    assert k == 2  # 1.0 -> 0.02 -> 4e-4; the next would give 8e-6 < 1e-4
    assert T == pytest.approx(0.02 * 0.02, rel=1e-12)
    d1, d2 = np.linalg.norm(ps[1]), np.linalg.norm(ps[2])
    want = 0.98 / d1 ** 2 + 0.98 * 0.02 ** 2 / d2 ** 2
    assert q[4] == pytest.approx(want, rel=1e-12)


# --------------------------------------------------------------------------
# projection (3DGS EWA convention, Sec. 3) against library routines
# --------------------------------------------------------------------------

def _conic_at(sc, g=0):
    sp = ora.project(sc, 0)[g]
    return sp, np.array([[sp[SP["CA"]], sp[SP["CB"]]], [sp[SP["CB"]], sp[SP["CC"]]]])


@pytest.mark.parametrize("seed", range(4))
def test_projection_on_axis_rotated(seed):
    """On the optical axis the EWA Jacobian is diag(f/z) in x, y, so the 2D
    covariance is (f/z)^2 Sigma[:2,:2] + dilation I with Sigma = R S^2 R^T;
    R from scipy (quaternion w,x,y,z -> scipy's x,y,z,w)."""
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(4)
    s = np.exp(rng.normal(-3, 0.5, 3))
    z = rng.uniform(1, 3)
    sc = tiny_scene([[0, 0, z]], s, quats=[q])
    cam = sc.cameras[0]
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    Sig = R @ np.diag(s ** 2) @ R.T
    S2 = (cam.fx / z) ** 2 * Sig[:2, :2] + 0.3 * np.eye(2)
    sp, conic = _conic_at(sc)
    np.testing.assert_allclose(conic, np.linalg.inv(S2), rtol=1e-10)
    assert sp[SP["U"]] == pytest.approx(cam.cx) and sp[SP["V"]] == pytest.approx(cam.cy)
    ev = np.linalg.eigvalsh(S2)
    assert sp[SP["RAD"]] == math.ceil(3 * math.sqrt(ev[-1]))


@pytest.mark.parametrize("pos", [[0.3, -0.2, 1.5], [-0.6, 0.4, 2.2], [0.05, 0.5, 1.1]])
def test_projection_off_axis_isotropic(pos):
    """Isotropic Sigma = s^2 I off axis: Sigma_2D = s^2 J J^T + dilation I
    with J the perspective Jacobian [[f/z, 0, -f x/z^2], [0, f/z, -f y/z^2]]."""
    s = 0.04
    sc = tiny_scene([pos], s)
    cam = sc.cameras[0]
    x, y, z = pos
    J = np.array([[cam.fx / z, 0, -cam.fx * x / z ** 2], [0, cam.fy / z, -cam.fy * y / z ** 2]])
    S2 = s * s * J @ J.T + 0.3 * np.eye(2)
    sp, conic = _conic_at(sc)
    np.testing.assert_allclose(conic, np.linalg.inv(S2), rtol=1e-10)
    assert sp[SP["U"]] == pytest.approx(cam.fx * x / z + cam.cx, rel=1e-14)
    assert sp[SP["V"]] == pytest.approx(cam.fy * y / z + cam.cy, rel=1e-14)
    assert sp[SP["Z"]] == pytest.approx(z)
    assert sp[SP["D"]] == pytest.approx(math.sqrt(x * x + y * y + z * z))


def test_moved_camera_uses_distance_to_optical_centre():
    """Falloff and phase use the distance to the optical centre o = -R^T t
    (Sec. 3), not the view depth; the view depth orders Gaussians."""
    R = Rotation.from_euler("xyz", [0.1, -0.2, 0.3]).as_matrix()
    centre = np.array([0.4, -0.3, -0.5])
    rt = np.concatenate([R, (-R @ centre)[:, None]], 1)
    x = np.array([0.2, 0.1, 2.0])
    sc = tiny_scene([x], 0.05, world_to_cam=rt)
    sp = ora.project(sc, 0)[0]
    p = R @ x + rt[:, 3]
    assert sp[SP["Z"]] == pytest.approx(p[2], rel=1e-14)
    assert sp[SP["D"]] == pytest.approx(np.linalg.norm(x - centre), rel=1e-14)
    d = np.linalg.norm(x - centre)
    assert sp[SP["FEAT"] + 2] == pytest.approx(1.0 / d ** 2, rel=1e-13)
    psi = 4 * math.pi * d * 30e6 / C_LIGHT
    assert sp[SP["FEAT"]] == pytest.approx(math.sin(psi) / d ** 2, rel=1e-12)
    assert sp[SP["FEAT"] + 1] == pytest.approx(math.cos(psi) / d ** 2, rel=1e-12)


def test_cubic_trajectory_and_displacement():
    """x(t) = mu + c1 t + c2 t^2 + c3 t^3 + delta_b (deformation step)."""
    mu = np.array([0.1, 0.2, 2.0])
    c = np.array([[0.3, -0.1, 0.2], [0.05, 0.4, -0.3], [-0.2, 0.1, 0.1]])
    delta = np.array([[[0.0, 0.0, 0.0]], [[0.01, -0.02, 0.03]]])
    times = (0.25, 0.8)
    sc = tiny_scene([mu], 0.05, coeffs=c[None], times=times, delta=delta)
    cam = sc.cameras[0]
    for b, t in enumerate(times):
        x = mu + c[0] * t + c[1] * t * t + c[2] * t ** 3 + delta[b, 0]
        sp = ora.project(sc, b)[0]
        assert sp[SP["U"]] == pytest.approx(cam.fx * x[0] / x[2] + cam.cx, rel=1e-13)
        assert sp[SP["V"]] == pytest.approx(cam.fy * x[1] / x[2] + cam.cy, rel=1e-13)
        assert sp[SP["D"]] == pytest.approx(np.linalg.norm(x), rel=1e-14)


def test_pixel_weight_matches_gaussian_density():
    """alpha at an off-centre pixel equals o exp(-1/2 d^T Sigma_2D^-1 d)
    (library inverse of the closed-form on-axis covariance)."""
    q = [0.9, 0.2, -0.3, 0.25]
    s = np.array([0.08, 0.03, 0.05])
    z = 1.5
    sc = tiny_scene([[0, 0, z]], s, quats=[q], opacity=[0.6], amplitude=[z * z])
    cam = sc.cameras[0]
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    S2 = (cam.fx / z) ** 2 * (R @ np.diag(s ** 2) @ R.T)[:2, :2] + 0.3 * np.eye(2)
    for px, py in [(33, 30), (29, 35), (36, 34)]:
        dlt = np.array([cam.cx - (px + 0.5), cam.cy - (py + 0.5)])
        alpha = 0.6 * math.exp(-0.5 * dlt @ np.linalg.solve(S2, dlt))
        q_out, T, k = _render_px(sc, px, py)
        if alpha >= 1 / 255:
            assert q_out[4] == pytest.approx(alpha, rel=1e-12)  # A = 1
            assert T == pytest.approx(1 - alpha, rel=1e-12)


# --------------------------------------------------------------------------
# binning (integer work) by brute force
# --------------------------------------------------------------------------

@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (16, 32)])
def test_binning_brute_force(tile):
    """Every (Gaussian, tile) pair tested against the FP32 rectangle; the
    per-tile lists ordered by (depth bits, index) equal the oracle's."""
    rng = np.random.default_rng(7)
    B, n, W, H = 2, 300, 100, 70
    u = rng.uniform(-20, W + 20, (B, n)).astype(np.float32)
    v = rng.uniform(-20, H + 20, (B, n)).astype(np.float32)
    r = rng.integers(0, 30, (B, n)).astype(np.int32)
    z = rng.uniform(0.3, 3, (B, n)).astype(np.float32)
    z[0, 5] = z[0, 6]  # an exact depth tie, broken by index
    keys, vals, ranges = ora.bin_f32(u, v, r, z, W, H, *tile)
    tw, th = np.float32(tile[0]), np.float32(tile[1])
    tx_n, ty_n = -(-W // tile[0]), -(-H // tile[1])
    idx = 0
    for b in range(B):
        for ty in range(ty_n):
            for tx in range(tx_n):
                members = []
                for g in range(n):
                    if r[b, g] <= 0:
                        continue
                    rf = np.float32(r[b, g])
                    x0 = np.floor(np.float32(u[b, g] - rf) / tw)
                    x1 = np.floor(np.float32(u[b, g] + rf) / tw) + 1
                    y0 = np.floor(np.float32(v[b, g] - rf) / th)
                    y1 = np.floor(np.float32(v[b, g] + rf) / th) + 1
                    if max(x0, 0) <= tx < min(x1, tx_n) and max(y0, 0) <= ty < min(y1, ty_n):
                        members.append((z[b, g].view(np.uint32), g))
                members.sort()
                t = b * tx_n * ty_n + ty * tx_n + tx
                assert ranges[t, 0] == idx
                for zb, g in members:
                    assert vals[idx] == g
                    assert keys[idx] == (np.uint64(t) << np.uint64(32)) | np.uint64(zb)
                    idx += 1
                assert ranges[t, 1] == idx
    assert idx == len(vals)


# --------------------------------------------------------------------------
# gradients: analytic (Eq. S3 + complex-step projection Jacobian) vs FD
# --------------------------------------------------------------------------

def _fd_scene(seed, n=6, W=24, H=20, freqs=(30e6,), frames=2):
    from paper_2505_05356_gb300 import scenes
    rng = np.random.default_rng(seed)
    cam = scenes.pinhole(W, H)
    z = rng.uniform(1.0, 2.5, n)
    pos = np.stack([rng.uniform(-0.3, 0.3, n) * z, rng.uniform(-0.3, 0.3, n) * z, z], 1)
    s = np.exp(rng.normal(-2.2, 0.3, (n, 3)))
    q = rng.standard_normal((n, 4))
    c = rng.normal(0, 0.05, (n, 3, 3))
    delta = rng.normal(0, 0.01, (frames, n, 3))
    sc = tiny_scene(pos, s, quats=q, opacity=rng.uniform(0.2, 0.9, n),
                    amplitude=rng.uniform(0.3, 1.0, n), width=W, height=H,
                    freqs=freqs, coeffs=c, times=tuple(np.linspace(0.1, 0.9, frames)),
                    delta=delta, bg=rng.uniform(-1, 1, len(freqs) * 4 + 1))
    return sc


def _loss(sc, dout, params):
    out, tf, amb, nc = ora.render(sc, params=params)
    return float(np.sum(out * dout)), amb


def _check_bg_by_differences(sc, dout, g):
    """dL/dbg against central differences of the oracle's own forward in a
    scene with Gaussians on every frame: Eq. 4 scales the background by the
    one-way T_N of each pixel (not T_N^2), and Eq. 5's mean depth has no
    background, so its entry must not move the loss at all.  The output is
    linear in bg (no decision depends on it), so the quotient is exact up to
    rounding."""
    bg0 = np.array(sc.bg, np.float64, copy=True)
    gbg = g["bg"]
    assert gbg.shape == bg0.shape
    tf = ora.render(sc)[1]
    assert tf.min() < 0.5  # T_N well below 1 somewhere: T_N and T_N^2 differ
    h = 1e-3
    for b in range(bg0.shape[0]):
        for c in range(bg0.shape[1]):
            vals = []
            for sgn in (1, -1):
                sc.bg = bg0.copy()
                sc.bg[b, c] += sgn * h
                vals.append(_loss(sc, dout, ora.Params(sc))[0])
            fd = (vals[0] - vals[1]) / (2 * h)
            assert gbg[b, c] == pytest.approx(fd, rel=1e-8, abs=1e-9 * (1 + abs(fd))), (b, c)
    sc.bg = bg0


@pytest.mark.parametrize("seed,freqs", [(0, (30e6,)), (1, (30e6, 80e6)), (2, (20e6,))])
def test_gradient_matches_central_differences(seed, freqs):
    sc = _fd_scene(seed, freqs=freqs)
    rng = np.random.default_rng(100 + seed)
    dout = rng.standard_normal((sc.frames, sc.n_channels, sc.height, sc.width))
    g = ora.backward(sc, dout)
    base = ora.Params(sc)
    L0, _ = _loss(sc, dout, base)
    names = ["means", "coeffs", "scales", "quats", "opacity", "amplitude", "delta"]
    checked = 0
    for name in names:
        arr = getattr(base, name)
        flat = arr.reshape(-1)
        gflat = g[name].reshape(-1)
        for i in range(flat.size):
            h = 1e-6 * max(1.0, abs(flat[i]))
            vals = []
            for sgn in (1, -1):
                P = ora.Params(sc)
                getattr(P, name).reshape(-1)[i] = flat[i] + sgn * h
                L, amb = _loss(sc, dout, P)
                # a discrete decision (rect, skip, stop, clamp) inside the step
                # makes the difference quotient meaningless; such a coordinate
                # is excluded (the random scenes keep them rare)
                vals.append((L, amb))
            fd = (vals[0][0] - vals[1][0]) / (2 * h)
            # discontinuity check: one-sided slopes must agree
            fr = (vals[0][0] - L0) / h
            fl = (L0 - vals[1][0]) / h
            if abs(fr - fl) > 1e-3 * (abs(fd) + 1e-3):
                continue
            assert gflat[i] == pytest.approx(fd, rel=2e-5, abs=2e-6 * (1 + abs(fd))), (name, i)
            checked += 1
    assert checked > 150
    _check_bg_by_differences(sc, dout, g)


def test_s3_recursion_against_direct_derivative():
    """Eq. S3 on one pixel: the recursion's d q / d alpha_k equals the
    derivative of sum_j alpha_j q_j T_j^2 + bg T_N written out directly."""
    rng = np.random.default_rng(5)
    K = 7
    a = rng.uniform(0.05, 0.6, K)
    q = rng.standard_normal(K)
    bg = 0.37

    def value(al):
        T, s = 1.0, 0.0
        for j in range(K):
            s += al[j] * q[j] * T * T
            T *= 1 - al[j]
        return s + bg * T

    # recursion as stated in the supplement (squared factors) + bg term
    T = np.cumprod(np.concatenate([[1.0], 1 - a]))[:K]
    Tn = np.prod(1 - a)
    acc, grads = 0.0, np.zeros(K)
    for k in range(K - 1, -1, -1):
        grads[k] = T[k] ** 2 * (q[k] + 2 * (a[k] - 1) * acc) - bg * Tn / (1 - a[k])
        acc = a[k] * q[k] + (1 - a[k]) ** 2 * acc
    for k in range(K):
        h = 1e-7
        ap, am = a.copy(), a.copy()
        ap[k] += h
        am[k] -= h
        assert grads[k] == pytest.approx((value(ap) - value(am)) / (2 * h), rel=1e-7)
    # and the oracle's 2D opacity gradient for the same stack of Gaussians
    cam = tiny_scene([[0, 0, 1]], 0.1).cameras[0]
    zs = np.linspace(1.0, 2.0, K)
    pos = [at_pixel(cam, 12.5, 9.5, z) for z in zs]
    ds = np.array([np.linalg.norm(p) for p in pos])
    sc = tiny_scene(pos, 0.02, opacity=a, amplitude=q * ds ** 2,
                    bg=[0, 0, 0, 0, bg])
    dout = np.zeros((1, 5, 64, 64))
    dout[0, 4, 9, 12] = 1.0
    g = ora.backward(sc, dout, want_2d=True)
    # d L / d o_k = d L / d alpha_k * G_k with G_k = 1 at the centre
    np.testing.assert_allclose(g["g2d"][0][:, 5], grads, rtol=1e-10, atol=1e-13)


# --------------------------------------------------------------------------
# extra channels: phasor (Eq. 3) and mean depth (Eq. 5)
# --------------------------------------------------------------------------

def _consts(**kw):
    from paper_2505_05356_gb300 import scenes
    return scenes.Consts(**kw)


def test_phasor_and_depth_single_and_two_gaussians():
    """One opaque Gaussian: phasor = 2 (0.99 A) exp(i psi) + p_bg T_N (Eq. 3)
    and mean depth = 0.99 d (Eq. 5, one-way T).  Two Gaussians: the depth
    weights are alpha_1 and alpha_2 (1 - alpha_1) -- one-way, unlike the
    squared transmittance of the C-ToF channels."""
    cam = tiny_scene([[0, 0, 1]], 0.1).cameras[0]
    p = np.array(at_pixel(cam, 25.5, 18.5, 1.0))
    d = 2.3
    pos = p / np.linalg.norm(p) * d
    bg = np.array([0.1, 0.2, 0.3, 0.4, -0.3, 0.7, -0.2, 5.0])  # last: depth (unused)
    sc = tiny_scene([pos], 0.03, opacity=[0.9999], amplitude=[0.8], bg=bg,
                    consts=_consts(phasor=True, depth=True))
    q, T, k = _render_px(sc, 25, 18)
    assert q.shape == (8,) and k == 1
    A = 0.8 / d ** 2
    psi = 4 * math.pi * d * 30e6 / C_LIGHT
    re, im = q[5] - 0.01 * bg[5], q[6] - 0.01 * bg[6]
    assert math.hypot(re, im) == pytest.approx(2 * 0.99 * A, rel=1e-12)
    assert math.atan2(im, re) % (2 * math.pi) == pytest.approx(psi % (2 * math.pi), abs=1e-12)
    assert q[7] == pytest.approx(0.99 * d, rel=1e-12)
    # two Gaussians on the pixel
    pa, pb = at_pixel(cam, 20.5, 30.5, 1.2), at_pixel(cam, 20.5, 30.5, 2.5)
    sc2 = tiny_scene([pb, pa], 0.03, opacity=[0.7, 0.4], consts=_consts(depth=True))
    q2, T2, k2 = _render_px(sc2, 20, 30)
    d1, d2 = np.linalg.norm(pa), np.linalg.norm(pb)
    assert q2[5] == pytest.approx(0.4 * d1 + 0.7 * (1 - 0.4) * d2, rel=1e-12)


def test_phasor_equals_quad_differences():
    """With a common bias on each quad pair the phasor is the quad
    differences of Sec. 2: Re = Q_pi/2 - Q_3pi/2, Im = Q_0 - Q_pi."""
    from paper_2505_05356_gb300 import scenes
    sc = scenes.make_scene("static_1k", 13, n=300, width=40, height=32, phasor=True)
    sc.sensor.offsets_rad = list(GOLDEN["phase_offsets_rad"]["value"])
    sc.bg[:] = 0.0
    out, tf, _, _ = ora.render(sc)
    np.testing.assert_allclose(out[0, 5], out[0, 1] - out[0, 3], atol=1e-12)
    np.testing.assert_allclose(out[0, 6], out[0, 0] - out[0, 2], atol=1e-12)


@pytest.mark.parametrize("seed", [7, 8])
def test_gradient_with_phasor_and_depth_matches_central_differences(seed):
    sc = _fd_scene(seed, n=5, freqs=(30e6, 80e6))
    sc.consts = _consts(phasor=True, depth=True)
    C = ora.n_channels(sc)
    assert C == 8 + 1 + 4 + 1
    sc.bg = np.random.default_rng(seed).uniform(-1, 1, (sc.frames, C))
    rng = np.random.default_rng(200 + seed)
    dout = rng.standard_normal((sc.frames, C, sc.height, sc.width))
    g = ora.backward(sc, dout)
    base = ora.Params(sc)
    L0, _ = _loss(sc, dout, base)
    checked = 0
    for name in ["means", "opacity", "amplitude", "scales", "quats", "coeffs"]:
        flat = getattr(base, name).reshape(-1)
        for i in range(flat.size):
            h = 1e-6 * max(1.0, abs(flat[i]))
            vals = []
            for sgn in (1, -1):
                P = ora.Params(sc)
                getattr(P, name).reshape(-1)[i] = flat[i] + sgn * h
                vals.append(_loss(sc, dout, P)[0])
            fd = (vals[0] - vals[1]) / (2 * h)
            if abs((vals[0] - L0) / h - (L0 - vals[1]) / h) > 1e-3 * (abs(fd) + 1e-3):
                continue
            assert g[name].reshape(-1)[i] == pytest.approx(fd, rel=2e-5, abs=2e-6 * (1 + abs(fd)))
            checked += 1
    assert checked > 80
    _check_bg_by_differences(sc, dout, g)
    assert np.all(g["bg"][:, C - 1] == 0.0)  # Eq. 5: no background in the mean depth


# --------------------------------------------------------------------------
# view-dependent reflectivity from spherical harmonics (Sec. 3)
# --------------------------------------------------------------------------

def _sh_scipy(l_index, x, y, z):
    """Real SH without the Condon-Shortley phase, from scipy's complex
    Y_l^m: m > 0 -> sqrt2 (-1)^m Re Y_l^m, m < 0 -> sqrt2 (-1)^m Im Y_l^|m|."""
    from scipy.special import sph_harm_y
    l = int(math.isqrt(l_index))
    m = l_index - l * l - l
    theta = math.acos(max(-1.0, min(1.0, z)))
    phi = math.atan2(y, x)
    if m == 0:
        return float(np.real(sph_harm_y(l, 0, theta, phi)))
    c = sph_harm_y(l, abs(m), theta, phi)
    sgn = -1.0 if abs(m) % 2 else 1.0
    return math.sqrt(2.0) * sgn * float(np.real(c) if m > 0 else np.imag(c))


def test_sh_basis_orthonormal_by_quadrature():
    """Gauss-Legendre in cos(theta) x uniform phi integrates products of
    degree <= 6 exactly: the 16 basis functions are orthonormal."""
    xs, ws = np.polynomial.legendre.leggauss(8)
    nphi = 16
    Y = []
    wts = []
    for ct, w in zip(xs, ws):
        st = math.sqrt(1.0 - ct * ct)
        for j in range(nphi):
            ph = 2.0 * math.pi * j / nphi
            x, y, z = st * math.cos(ph), st * math.sin(ph), ct
            Y.append([ora.sh_basis(l, x, y, z) for l in range(16)])
            wts.append(w * 2.0 * math.pi / nphi)
    Y = np.asarray(Y)
    G = Y.T @ (Y * np.asarray(wts)[:, None])
    np.testing.assert_allclose(G, np.eye(16), atol=1e-13)


def test_sh_basis_matches_scipy_real_form():
    rng = np.random.default_rng(3)
    for _ in range(20):
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        for l in range(16):
            assert ora.sh_basis(l, *v) == pytest.approx(_sh_scipy(l, *v), abs=1e-13), l


@pytest.mark.parametrize("n_sh", [1, 4, 9, 16])
def test_sh_reflectivity_uses_world_direction_from_optical_centre(n_sh):
    """A = s r / d^2 with r = max(0, 0.5 + sum c_l Y_l(dir)), dir the unit
    vector from the optical centre to the centre in world coordinates (a
    rotated, shifted camera separates world and camera frames)."""
    R = Rotation.from_euler("xyz", [0.2, -0.3, 0.25]).as_matrix()
    centre = np.array([0.3, -0.2, -0.4])
    rt = np.concatenate([R, (-R @ centre)[:, None]], 1)
    rng = np.random.default_rng(n_sh)
    xs = [centre + R.T @ np.array([0.1, -0.05, 2.0]),
          centre + R.T @ np.array([-0.2, 0.1, 1.5])]
    sh = rng.normal(0.0, 0.4, (2, n_sh))
    sh[1, 0] = -3.0  # negative before the clamp: r = 0
    sc = tiny_scene(xs, 0.05, world_to_cam=rt, sh=sh, source_intensity=1.7)
    sp = ora.project(sc, 0)
    for k in range(2):
        d = np.linalg.norm(xs[k] - centre)
        u = (xs[k] - centre) / d
        r = 0.5 + sum(sh[k, l] * _sh_scipy(l, *u) for l in range(n_sh))
        r = max(r, 0.0)
        assert sp[k, SP["FEAT"] + 2] == pytest.approx(1.7 * r / d ** 2, rel=1e-12, abs=1e-15)
    assert sp[1, SP["FEAT"] + 2] == 0.0


def test_sh_degree_zero_equals_scalar_amplitude():
    """n_sh = 1 with c_0 = (r - 0.5) / Y_0 reproduces the scalar model."""
    rng = np.random.default_rng(5)
    sc = _fd_scene(5, n=6, frames=1)
    out0, _, _, _ = ora.render(sc)
    sc.sh = ((sc.amplitude - 0.5) * 2.0 * math.sqrt(math.pi))[:, None]
    sc.amplitude = rng.uniform(0.0, 1.0, sc.n)  # ignored under SH
    out1, _, _, _ = ora.render(sc)
    np.testing.assert_allclose(out1, out0, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("seed,n_sh", [(11, 16), (12, 4)])
def test_gradient_with_sh_matches_central_differences(seed, n_sh):
    sc = _fd_scene(seed, n=5)
    R = Rotation.from_euler("xyz", [0.05, -0.1, 0.08]).as_matrix()
    centre = np.array([0.1, -0.05, -0.2])
    rt = np.concatenate([R, (-R @ centre)[:, None]], 1)
    for cam in sc.cameras:
        cam.world_to_cam = rt
    rng = np.random.default_rng(300 + seed)
    sc.sh = rng.normal(0.0, 0.2, (sc.n, n_sh))
    sc.sh[:, 0] = 0.8
    dout = rng.standard_normal((sc.frames, sc.n_channels, sc.height, sc.width))
    g = ora.backward(sc, dout)
    assert g["sh"].shape == (sc.n, n_sh)
    assert np.all(g["amplitude"] == 0.0)
    base = ora.Params(sc)
    L0, _ = _loss(sc, dout, base)
    checked = 0
    for name in ["sh", "means", "coeffs", "delta"]:
        arr = getattr(base, name)
        idx = [(k, l) for k in range(sc.n) for l in range(n_sh)] if name == "sh" else \
            list(range(arr.size))
        for i in idx:
            get = (lambda P: P.sh[i]) if name == "sh" else \
                (lambda P, name=name: getattr(P, name).reshape(-1)[i])
            x0 = get(base)
            h = 1e-6 * max(1.0, abs(x0))
            vals = []
            for sgn in (1, -1):
                P = ora.Params(sc)
                if name == "sh":
                    P.sh[i] = x0 + sgn * h
                else:
                    getattr(P, name).reshape(-1)[i] = x0 + sgn * h
                vals.append(_loss(sc, dout, P)[0])
            fd = (vals[0] - vals[1]) / (2 * h)
            if abs((vals[0] - L0) / h - (L0 - vals[1]) / h) > 1e-3 * (abs(fd) + 1e-3):
                continue
            ga = g[name][i] if name == "sh" else g[name].reshape(-1)[i]
            assert ga == pytest.approx(fd, rel=2e-5, abs=2e-6 * (1 + abs(fd))), (name, i)
            checked += 1
    assert checked > 60


# --------------------------------------------------------------------------
# asynchronous raw capture and piecewise-linear motion (Sec. 3, Eq. 7)
# --------------------------------------------------------------------------

def test_eq7_interpolates_positions_between_timesteps():
    """Positions at t in [t0, t1] are the linear interpolation of those at t0
    and t1 (numpy polynomial evaluation of the trajectory at both ends); a
    linear trajectory is reproduced exactly, t = t0 gives x(t0)."""
    mu = np.array([0.1, -0.2, 2.0])
    c = np.array([[0.3, -0.1, 0.2], [0.5, 0.4, -0.3], [-0.6, 0.2, 0.4]])
    t0, t1 = 0.2, 0.6
    times = (0.2, 0.35, 0.5, 0.6)
    sc = tiny_scene([mu], 0.05, coeffs=c[None], times=times,
                    interp_times=[[t0, t1]] * len(times))
    cam = sc.cameras[0]

    def traj(t):
        return mu + c[0] * t + c[1] * t ** 2 + c[2] * t ** 3

    for b, t in enumerate(times):
        x = traj(t0) + (t - t0) / (t1 - t0) * (traj(t1) - traj(t0))
        sp = ora.project(sc, b)[0]
        assert sp[SP["U"]] == pytest.approx(cam.fx * x[0] / x[2] + cam.cx, rel=1e-13)
        assert sp[SP["V"]] == pytest.approx(cam.fy * x[1] / x[2] + cam.cy, rel=1e-13)
        assert sp[SP["D"]] == pytest.approx(np.linalg.norm(x), rel=1e-14)
    # a mid-interval frame differs from the exact trajectory for a curved path
    exact = tiny_scene([mu], 0.05, coeffs=c[None], times=(0.35,))
    assert abs(ora.project(exact, 0)[0][SP["D"]] - ora.project(sc, 1)[0][SP["D"]]) > 1e-4
    # a straight path is reproduced exactly
    c_lin = c.copy()
    c_lin[1:] = 0.0
    lin = tiny_scene([mu], 0.05, coeffs=c_lin[None], times=(0.35,), interp_times=[[t0, t1]])
    lin_exact = tiny_scene([mu], 0.05, coeffs=c_lin[None], times=(0.35,))
    np.testing.assert_allclose(ora.project(lin, 0), ora.project(lin_exact, 0), rtol=1e-13,
                               atol=1e-15)


def test_async_frame_equals_matching_channel_of_synchronous_quartet():
    """A frame that samples one offset phi (P = 1, frame phase phi) equals the
    channel phi of a synchronous four-offset frame at the same time."""
    sc4 = _fd_scene(21, n=6, frames=1)
    offs = [0.0, math.pi / 2, math.pi, 3 * math.pi / 2]
    sc4.sensor.offsets_rad = offs
    q4, tf4, _, _ = ora.render(sc4)
    for j, phi in enumerate(offs):
        sc1 = _fd_scene(21, n=6, frames=1)
        sc1.sensor.offsets_rad = [0.0]
        sc1.bg = np.stack([sc4.bg[:, j], sc4.bg[:, 4]], 1)
        sc1.frame_phase = np.array([phi])
        q1, tf1, _, _ = ora.render(sc1)
        np.testing.assert_allclose(q1[0, 0], q4[0, j], rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(q1[0, 1], q4[0, 4], rtol=1e-13, atol=1e-15)
        np.testing.assert_array_equal(tf1, tf4)


@pytest.mark.parametrize("seed", [31, 32])
def test_gradient_async_interpolated_matches_central_differences(seed):
    sc = _fd_scene(seed, n=5, frames=3)
    sc.sensor.offsets_rad = [0.0]
    sc.frame_phase = np.array([0.0, math.pi / 2, math.pi])
    sc.interp_times = np.array([[0.1, 0.7], [0.1, 0.7], [0.1, 0.7]])
    sc.bg = np.random.default_rng(seed).uniform(-1, 1, (sc.frames, 2))
    rng = np.random.default_rng(400 + seed)
    dout = rng.standard_normal((sc.frames, sc.n_channels, sc.height, sc.width))
    g = ora.backward(sc, dout)
    base = ora.Params(sc)
    L0, _ = _loss(sc, dout, base)
    checked = 0
    for name in ["means", "coeffs", "delta", "opacity", "amplitude"]:
        flat = getattr(base, name).reshape(-1)
        for i in range(flat.size):
            h = 1e-6 * max(1.0, abs(flat[i]))
            vals = []
            for sgn in (1, -1):
                P = ora.Params(sc)
                getattr(P, name).reshape(-1)[i] = flat[i] + sgn * h
                vals.append(_loss(sc, dout, P)[0])
            fd = (vals[0] - vals[1]) / (2 * h)
            if abs((vals[0] - L0) / h - (L0 - vals[1]) / h) > 1e-3 * (abs(fd) + 1e-3):
                continue
            assert g[name].reshape(-1)[i] == pytest.approx(fd, rel=2e-5, abs=2e-6 * (1 + abs(fd)))
            checked += 1
    assert checked > 60


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_squared_transmittance_telescopes_for_any_scene(seed):
    """The weights of the round trip telescope for any scene: with T_{k+1} =
    T_k (1 - alpha_k), alpha_k (2 - alpha_k) T_k^2 = T_k^2 - T_{k+1}^2, so
    sum_k alpha_k (2 - alpha_k) T_k^2 = 1 - T_N^2 (Eq. 4's T_k^2; the early
    stop only ends the sum).  Checked on the oracle's instrumented walk of
    pixels with dozens of contributors."""
    from paper_2505_05356_gb300 import scenes
    sc = scenes.make_scene("static_1k", seed, n=1500, width=48, height=40)
    splats = ora.project(sc, 0)
    rng = np.random.default_rng(seed)
    deep = 0
    for x, y in rng.integers(0, [48, 40], size=(40, 2)):
        a, T, TN = ora.pixel_steps(sc, 0, x, y, splats=splats)
        if len(a) == 0:
            assert TN == 1.0
            continue
        deep += len(a) >= 20
        np.testing.assert_allclose(T[1:], T[:-1] * (1 - a[:-1]), rtol=1e-15)
        assert T[0] == 1.0 and TN == pytest.approx(T[-1] * (1 - a[-1]), rel=1e-15)
        assert float(np.sum(a * (2 - a) * T * T)) == pytest.approx(1 - TN * TN, abs=1e-13)
    assert deep >= 5


# --------------------------------------------------------------------------
# every valid result of an ambiguous pixel (the walk re-run with its
# near-threshold decisions taken the other way)
# --------------------------------------------------------------------------

def _alts_at(sc, x, y):
    k = sc.consts
    r = ora.render_tiles(sc, 0, [(x // k.tile_w, y // k.tile_h)], eps=ora.EPS_F32)
    i = int(np.flatnonzero((r["pix"][:, 0] == x) & (r["pix"][:, 1] == y))[0])
    return r, i


def _quads(sp, weights, T, bg, offsets):
    """Eq. 4 written out: Q_j = sum_k w_k (A sin psi_k cos phi_j + A cos psi_k
    sin phi_j) + bg_j T, ambient = sum_k w_k A_k + bg_amb T."""
    S = ora.SP
    q = [sum(w * (sp[g, S["FEAT"]] * np.cos(ph) + sp[g, S["FEAT"] + 1] * np.sin(ph))
             for g, w in weights) + bg[j] * T for j, ph in enumerate(offsets)]
    q.append(sum(w * sp[g, S["FEAT"] + 2] for g, w in weights) + bg[len(offsets)] * T)
    return np.array(q)


def test_alternatives_of_a_near_depth_tie_are_both_orders():
    """Two Gaussians on one pixel (0.1 px off its centre, so no power > 0
    question arises) at depths 2 relative 2.5e-7 apart (closer than single
    precision resolves): the pixel is flagged, and its valid results are
    exactly the two compositing orders, alpha_a then alpha_b and the reverse
    (weights alpha T^2, T the product of (1 - alpha))."""
    cam = tiny_scene([[0, 0, 1]], 0.1).cameras[0]
    pa = np.array(at_pixel(cam, 20.6, 30.4, 2.0))
    pb = pa * (1 + 2.5e-7)
    bg = np.array([0.3, -0.2, 0.1, 0.4, 0.25])
    sc = tiny_scene([pa, pb], 0.05, opacity=[0.6, 0.3], bg=bg)
    r, i = _alts_at(sc, 20, 30)
    assert r["ambig"][i] & ora.AMB["ORDER"]
    alts = r["alts"][i]
    assert alts.shape[0] == 2
    sp = ora.project(sc, 0)
    S = ora.SP
    al = [min(0.99, sp[g, S["OPA"]] * np.exp(-0.5 * (sp[g, S["CA"]] * (sp[g, S["U"]] - 20.5) ** 2 +
                                                       sp[g, S["CC"]] * (sp[g, S["V"]] - 30.5) ** 2)
                                                - sp[g, S["CB"]] * (sp[g, S["U"]] - 20.5) *
                                                (sp[g, S["V"]] - 30.5)))
          for g in (0, 1)]
    offs = sc.sensor.offsets_rad
    T = (1 - al[0]) * (1 - al[1])
    ab = _quads(sp, [(0, al[0]), (1, al[1] * (1 - al[0]) ** 2)], T, bg, offs)
    ba = _quads(sp, [(1, al[1]), (0, al[0] * (1 - al[1]) ** 2)], T, bg, offs)
    np.testing.assert_allclose(alts[0], ab, rtol=1e-12, atol=1e-14)  # nominal first: a in front
    np.testing.assert_allclose(alts[1], ba, rtol=1e-12, atol=1e-14)
    np.testing.assert_array_equal(alts[0], r["out"][i])


def test_alternatives_at_the_alpha_floor_composite_or_skip():
    """A Gaussian of opacity alpha_min 0.004 px from the pixel centre (its
    alpha there is below alpha_min by ~5e-6 relative) behind an ordinary one:
    the pixel is flagged, and its valid results are without it (the nominal
    walk) and with it."""
    cam = tiny_scene([[0, 0, 1]], 0.1).cameras[0]
    pa = np.array(at_pixel(cam, 12.7, 9.4, 1.5))
    pb = np.array(at_pixel(cam, 12.504, 9.5, 2.5))
    bg = np.array([0.3, -0.2, 0.1, 0.4, 0.25])
    sc = tiny_scene([pa, pb], 0.05, opacity=[0.5, 1.0 / 255.0], bg=bg)
    r, i = _alts_at(sc, 12, 9)
    assert r["ambig"][i] & ora.AMB["ALPHA_MIN"]
    alts = r["alts"][i]
    sp = ora.project(sc, 0)
    S = ora.SP

    def alpha(g):
        dx, dy = sp[g, S["U"]] - 12.5, sp[g, S["V"]] - 9.5
        return sp[g, S["OPA"]] * np.exp(-0.5 * (sp[g, S["CA"]] * dx * dx + sp[g, S["CC"]] * dy * dy)
                                        - sp[g, S["CB"]] * dx * dy)
    a0, a1 = alpha(0), alpha(1)
    offs = sc.sensor.offsets_rad
    without = _quads(sp, [(0, a0)], 1 - a0, bg, offs)
    with_ = _quads(sp, [(0, a0), (1, a1 * (1 - a0) ** 2)], (1 - a0) * (1 - a1), bg, offs)
    got = sorted(alts.tolist(), key=lambda q: q[0])
    want = sorted([without.tolist(), with_.tolist()], key=lambda q: q[0])
    assert len(got) == 2
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(alts[0], without, rtol=1e-12, atol=1e-14)  # nominal: skipped


def test_no_alternatives_without_a_near_threshold_decision():
    sc = tiny_scene([at_pixel(tiny_scene([[0, 0, 1]], 0.1).cameras[0], 30.7, 30.4, 2.0)], 0.05,
                    opacity=[0.7])
    r, i = _alts_at(sc, 30, 30)
    assert r["ambig"][i] == 0 and i not in r["alts"]
