"""Plain FP64 reference of the optimisation-loop steps (test infrastructure only).

Only the test-suite and the CPU-baseline leg of ``bench.py`` may import this
module; it shares nothing with the CUDA path.

* ``splitmix64_stream`` -- the SplitMix64 generator (Steele, Lea and Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014; the 64-bit
  finaliser constants of Vigna's public-domain splitmix64.c), run
  sequentially: state += 0x9E3779B97F4A7C15, output = mix(state).
* ``background_sample`` -- the per-iteration random background of Sec. 4
  ("Random background": a fresh background, uniform in [-1, 1], at every
  optimisation iteration): value = 2 u - 1 with u the top 24 bits of the
  generator's output times 2^-24, drawn in (iteration, channel) order.
* ``l2_loss`` -- the raw-sample L2 reconstruction term of the loss (Sec. 4,
  the L_q term of the total loss, Eq. 9, without SSIM): mean of squared residuals over the raw channels.
* ``adam_step`` -- Adam (Kingma and Ba, ICLR 2015, Algorithm 1) with the
  paper's betas and epsilon (Sec. 4, "Hyperparameters"), followed by a
  projection onto [lo, hi] that keeps the parameters valid for rendering.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def _mix64(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def splitmix64_stream(seed: int, count: int):
    """The first `count` outputs of SplitMix64 seeded with `seed`."""
    s = seed & MASK64
    out = []
    for _ in range(count):
        s = (s + GAMMA) & MASK64
        out.append(_mix64(s))
    return out


def background_sample(seed: int, iterations: int, n_bg: int) -> np.ndarray:
    """(iterations, n_bg) backgrounds: iteration s (1-based) takes outputs
    (s - 1) n_bg + 1 .. s n_bg of the stream."""
    raw = splitmix64_stream(seed, iterations * n_bg)
    u = np.array([(r >> 40) for r in raw], np.float64) * 2.0 ** -24
    return (2.0 * u - 1.0).reshape(iterations, n_bg)


def l2_loss(out: np.ndarray, target: np.ndarray, n_raw: int):
    """(loss, dL/dout) for out, target shaped (B, C, H, W): the mean of the
    squared residuals over channels [0, n_raw); the other channels get 0."""
    out = np.asarray(out, np.float64)
    target = np.asarray(target, np.float64)
    r = out[:, :n_raw] - target[:, :n_raw]
    M = r.size
    loss = float(np.sum(r * r) / M)
    g = np.zeros_like(out)
    g[:, :n_raw] = 2.0 * r / M
    return loss, g


def adam_step(param, grad, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-15,
              lo=-np.inf, hi=np.inf):
    """One Adam update at step t >= 1; returns (param, m, v) as new float64
    arrays."""
    g = np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    p = np.asarray(param, np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps)
    return np.clip(p, lo, hi), m, v
