"""Shared helpers of the GPU parity tests: run the CUDA path through the
binding on a seeded scene, and compare with the oracle's results."""
import numpy as np
import torch

from oracle import oracle as ora
from paper_2505_05356_gb300 import gftorf


def run_gpu(scene, dout=None, dtype=torch.float32, render_mode=0, capacity=None,
            grads=True, pixels_per_thread=0, flags=0):
    """Forward (and backward for dout) of the CUDA path on `scene`."""
    dev = "cuda"
    r = gftorf.Renderer(scene.n, scene.frames, scene.width, scene.height,
                        len(scene.sensor.freqs_hz), len(scene.sensor.offsets_rad),
                        tile=(scene.consts.tile_w, scene.consts.tile_h), dtype=dtype,
                        render_mode=render_mode,
                        max_instances=capacity, pixels_per_thread=pixels_per_thread,
                        flags=flags | gftorf.flags_from_scene(scene),
                        n_sh=getattr(scene, "n_sh", 0))
    p = gftorf.params_from_scene(scene, dev, dtype)
    fr = gftorf.frames_from_scene(scene)
    se = gftorf.sensor_from_scene(scene)
    co = gftorf.consts_from_scene(scene)
    bg = torch.as_tensor(scene.bg).to(dev, dtype).contiguous()
    if capacity is None:
        r.fit_capacity(p, fr, se, co, bg)
    r.preprocess(p, fr, se, co)
    out = r.render_fwd(bg)
    res = dict(renderer=r, out=out.double().cpu().numpy())
    tf, nl = r.pixel_state()
    res["tfinal"] = tf.double().cpu().numpy()
    res["nlast"] = nl.cpu().numpy()
    res["status"] = r.read_status()
    if dout is not None and grads:
        g = r.render_bwd(p, bg, torch.as_tensor(dout).to(dev, dtype).contiguous())
        torch.cuda.synchronize()
        res["grads"] = {k: v.double().cpu().numpy() for k, v in g.items()}
    return res


def forward_close(q_gpu, q_ora, amb, rel=1e-5, flag_mask=ora.AMB_VALUE):
    """Per-channel scaled relative error on the unambiguous pixels:
    |Q_gpu - Q_ora| <= rel * max(|Q_ora|, RMS_c).  Returns (ok, worst, n_flag)."""
    B, C = q_ora.shape[:2]
    keep = (amb & flag_mask) == 0  # (B, H, W)
    worst = 0.0
    for b in range(B):
        for c in range(C):
            o = q_ora[b, c]
            sig = np.sqrt(np.mean(o * o)) + 1e-300
            err = np.abs(q_gpu[b, c] - o) / np.maximum(np.abs(o), sig)
            e = err[keep[b]]
            if e.size:
                worst = max(worst, float(e.max()))
    return worst <= rel, worst, int((~keep).sum())


def match_alternatives(q_gpu, alts, sigma, rel=1e-5):
    """Smallest, over the valid oracle results `alts` (k, C) of one pixel, of
    the largest per-channel error |q_gpu - alt| / max(|alt|, sigma_c).  The
    pixel is correct when this is <= rel: single precision took each of its
    near-threshold decisions one of the two ways, and the result matches the
    oracle walk that took the same ones."""
    err = np.abs(q_gpu[None, :] - alts) / np.maximum(np.abs(alts), sigma[None, :])
    return float(err.max(axis=1).min())


def ambiguous_pixels_match(scene, b, q_gpu, q_ora, amb, rel=1e-5):
    """Every pixel of frame b with a value-changing ambiguity flag equals one
    of the oracle's valid results for it (the walk re-run with its
    near-threshold decisions taken the other way).  q_gpu, q_ora: (C, H, W);
    amb: (H, W).  Returns (flagged, worst best-match error, capped searches)."""
    C = q_ora.shape[0]
    sigma = np.sqrt((q_ora.reshape(C, -1) ** 2).mean(axis=1)) + 1e-300
    flagged = np.argwhere((amb & ora.AMB_VALUE) != 0)  # (y, x)
    if len(flagged) == 0:
        return 0, 0.0, 0
    k = scene.consts
    tiles = np.unique(np.stack([flagged[:, 1] // k.tile_w, flagged[:, 0] // k.tile_h], 1), axis=0)
    r = ora.render_tiles(scene, b, tiles, eps=ora.EPS_F32)
    index = {(int(x), int(y)): i for i, (x, y) in enumerate(r["pix"])}
    worst = 0.0
    for y, x in flagged:
        i = index[(int(x), int(y))]
        alts = r["alts"].get(i, r["out"][i:i + 1])
        worst = max(worst, match_alternatives(q_gpu[:, y, x], alts, sigma, rel))
    return len(flagged), worst, r["capped"]


def absent_groups(scene):
    """Gradient groups the CUDA path does not return for `scene` because the
    scene has no such parameter (static trajectories, no per-frame
    displacement, scalar reflectivity)."""
    out = set()
    for k in ("coeffs", "delta", "amplitude", "sh"):
        if getattr(scene, k, None) is None:
            out.add(k)
    return out


def grads_close(g_gpu, g_ora, rel=1e-3, absent=()):
    """Per parameter group: norm-wise relative error and elementwise error
    against max(|g|, RMS of the group).  Returns dict name -> (norm, elem).
    Every group of g_ora must be in g_gpu unless listed in `absent`."""
    out = {}
    for k, go in g_ora.items():
        if k not in g_gpu:
            assert k in absent, "gradient group %r missing from the CUDA path's result" % k
            continue
        gg = g_gpu[k].reshape(-1)
        go = np.asarray(go, np.float64).reshape(-1)
        nrm = np.linalg.norm(go)
        if nrm == 0:
            out[k] = (float(np.abs(gg).max()) if gg.size else 0.0, 0.0)
            continue
        rms = nrm / np.sqrt(go.size)
        out[k] = (float(np.linalg.norm(gg - go) / nrm),
                  float(np.max(np.abs(gg - go) / np.maximum(np.abs(go), rms))))
    return out
