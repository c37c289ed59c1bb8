"""FP64 reference of the deformation MLP (test infrastructure only).

Only the test-suite and the CPU-baseline leg of ``bench.py`` may import this
module; it shares nothing with the CUDA path.

The network of Sec. 4 ("MLP", "Initialization"): the offset of Gaussian k at
time t is delta_x = MLP(gamma(x_k / d_u), gamma(t)), with the positions
rescaled by the unambiguous range d_u (so they mostly lie in [0, 1]) and the
positional encoding gamma(p) = (p, sin(2^l pi p), cos(2^l pi p), l = 0..L-1)
with L_x = L_t = 10 frequencies; 8 hidden layers of 256 units with ReLU and a
linear head to the 3 offset components.

Layout fixed here and in the C ABI: the encoded input of row m = b N + g
(frame b, Gaussian g) is
  [x_0, x_1, x_2, then for l = 0..9: sin(2^l pi x_0..2), cos(2^l pi x_0..2),
   t, then for l = 0..9: sin(2^l pi t), cos(2^l pi t)]   (84 values)
zero-padded to 128.  The packed parameter vector is
  [W_0 (256 x 128), b_0 (256), W_1 (256 x 256), b_1, ..., W_7, b_7,
   W_head (3 x 256), b_head (3)]
with W row-major (out, in): layer out = W in + b.

Mixed precision of the tensor-core path (``bf16=True``): the operands of every
matrix product are rounded to bfloat16 (round to nearest even) -- weights,
the encoded input, hidden activations, the back-propagated pre-activation
gradients -- and products are summed exactly (here in double precision);
biases, the head's output and the encoding's gradient stay wide.
``bf16=False`` is the plain FP64 network.
"""
from __future__ import annotations

import math

import numpy as np

WIDTH = 256
DEPTH = 8
IN_PAD = 128
N_FREQ = 10
ENC_X = 3 * (1 + 2 * N_FREQ)   # 63
ENC_T = 1 + 2 * N_FREQ         # 21


def layer_shapes():
    """[(out, in)] of the 8 hidden layers and the head."""
    return [(WIDTH, IN_PAD)] + [(WIDTH, WIDTH)] * (DEPTH - 1) + [(3, WIDTH)]


def n_params() -> int:
    return sum(o * i + o for o, i in layer_shapes())


def unpack(theta):
    """Packed vector -> [(W, b)] (views)."""
    theta = np.asarray(theta, np.float64)
    out, at = [], 0
    for o, i in layer_shapes():
        W = theta[at:at + o * i].reshape(o, i)
        at += o * i
        b = theta[at:at + o]
        at += o
        out.append((W, b))
    return out


def pack(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in layers])


def to_bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    x32 = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = x32.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _scaled(means, inv_scale, single):
    if single:
        # the scaled positions as a single-precision implementation forms them
        # (one rounded product): the 2^9 pi of the top frequency turns their
        # rounding into phase differences far above a BF16 ulp, so the check
        # of such an implementation encodes the same single-precision inputs
        return (np.asarray(means, np.float32) * np.float32(inv_scale)).astype(np.float64)
    return np.asarray(means, np.float64) * inv_scale


def encode(means, times, inv_scale, single=False):
    """Encoded inputs (B * N, 128), row b N + g; single=True encodes the
    single-precision scaled positions."""
    means = np.asarray(means, np.float64)
    times = np.asarray(times, np.float64)
    N, B = means.shape[0], times.shape[0]
    x = _scaled(means, inv_scale, single)
    cols = [x]
    for l in range(N_FREQ):
        cols.append(np.sin(2.0 ** l * math.pi * x))
        cols.append(np.cos(2.0 ** l * math.pi * x))
    ex = np.concatenate(cols, 1)                      # (N, 63)
    rows = []
    for b in range(B):
        t = times[b]
        et = [t]
        for l in range(N_FREQ):
            et += [math.sin(2.0 ** l * math.pi * t), math.cos(2.0 ** l * math.pi * t)]
        enc = np.zeros((N, IN_PAD))
        enc[:, :ENC_X] = ex
        enc[:, ENC_X:ENC_X + ENC_T] = np.asarray(et)[None, :]
        rows.append(enc)
    return np.concatenate(rows, 0)


def encode_backward(d_enc, means, times, inv_scale, single=False):
    """dL/d(means) (N, 3), summed over the frames, from dL/d(encoded input)."""
    means = np.asarray(means, np.float64)
    N, B = means.shape[0], len(times)
    x = _scaled(means, inv_scale, single)
    g = np.zeros((N, 3))
    for b in range(B):
        d = np.asarray(d_enc[b * N:(b + 1) * N], np.float64)
        gx = d[:, 0:3].copy()
        for l in range(N_FREQ):
            w = 2.0 ** l * math.pi
            ds = d[:, 3 + 6 * l:6 + 6 * l]
            dc = d[:, 6 + 6 * l:9 + 6 * l]
            gx += w * (np.cos(w * x) * ds - np.sin(w * x) * dc)
        g += gx * inv_scale
    return g


def forward(theta, enc, bf16=True):
    """(delta (M, 3), cache) for encoded inputs enc (M, 128)."""
    r = to_bf16 if bf16 else (lambda a: np.asarray(a, np.float64))
    layers = unpack(theta)
    h = r(enc)
    acts = [h]
    for W, b in layers[:-1]:
        h = r(np.maximum(h @ r(W).T + b, 0.0))
        acts.append(h)
    Wh, bh = layers[-1]
    delta = h @ r(Wh).T + bh
    return delta, acts


def backward(theta, acts, d_delta, bf16=True):
    """(d_theta packed, d_enc (M, 128)) for dL/d(delta) (M, 3)."""
    r = to_bf16 if bf16 else (lambda a: np.asarray(a, np.float64))
    layers = unpack(theta)
    grads = []
    dz = r(d_delta)
    Wh, _ = layers[-1]
    grads.append((dz.T @ acts[-1], dz.sum(0)))
    dh = dz @ r(Wh)
    for li in range(DEPTH - 1, -1, -1):
        W, _ = layers[li]
        dz = r(dh * (acts[li + 1] > 0))
        grads.append((dz.T @ acts[li], dz.sum(0)))
        dh = dz @ r(W)
    grads.reverse()
    return pack(grads), dh
