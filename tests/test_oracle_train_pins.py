"""Pins of the optimisation-loop oracle (oracle/train.py) against published
values and closed forms: SplitMix64's first outputs for seed 0, Adam's first
two steps in closed form (Kingma and Ba, Algorithm 1), the L2 loss gradient
by central differences, and the background's range and moments."""
import math

import numpy as np
import pytest

from oracle import train


def test_splitmix64_published_outputs_seed0():
    # the first two outputs of SplitMix64 seeded with 0, as printed with
    # Vigna's splitmix64.c
    out = train.splitmix64_stream(0, 2)
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]


def test_background_range_moments_and_order():
    bg = train.background_sample(7, 400, 5)
    assert bg.shape == (400, 5)
    assert bg.min() >= -1.0 and bg.max() < 1.0
    assert abs(bg.mean()) < 0.05
    assert abs(np.mean(bg * bg) - 1.0 / 3.0) < 0.03  # U(-1, 1): E[x^2] = 1/3
    # values are exact multiples of 2^-23 (24-bit uniforms), float32-exact
    assert np.all(bg == bg.astype(np.float32))
    # iteration s continues the stream where iteration s - 1 stopped
    one = train.background_sample(7, 2, 5)
    flat = train.background_sample(7, 1, 10)
    np.testing.assert_array_equal(one.reshape(-1), flat.reshape(-1))


def test_adam_first_two_steps_closed_form():
    g1, g2 = np.array([0.3, -2.0, 1e-3]), np.array([-0.1, -1.0, 2e-3])
    p0 = np.array([1.0, 0.5, -0.25])
    lr, b1, b2, eps = 0.01, 0.9, 0.999, 1e-15
    p1, m, v = train.adam_step(p0, g1, 0, 0, 1, lr, b1, b2, eps)
    # step 1: m_hat = g, v_hat = g^2  ->  p1 = p0 - lr g / (|g| + eps)
    np.testing.assert_allclose(p1, p0 - lr * g1 / (np.abs(g1) + eps), rtol=1e-15)
    p2, m, v = train.adam_step(p1, g2, m, v, 2, lr, b1, b2, eps)
    m2 = (b1 * (1 - b1) * g1 + (1 - b1) * g2) / (1 - b1 ** 2)
    v2 = (b2 * (1 - b2) * g1 ** 2 + (1 - b2) * g2 ** 2) / (1 - b2 ** 2)
    np.testing.assert_allclose(p2, p1 - lr * m2 / (np.sqrt(v2) + eps), rtol=1e-14)


def test_adam_projection():
    p, _, _ = train.adam_step(np.array([0.001, 0.999]), np.array([1.0, -1.0]), 0, 0, 1, 0.01,
                              lo=1e-4, hi=1.0)
    np.testing.assert_array_equal(p, [1e-4, 1.0])


def test_l2_loss_value_and_central_differences():
    rng = np.random.default_rng(3)
    out = rng.standard_normal((2, 5, 3, 4))
    tgt = rng.standard_normal((2, 5, 3, 4))
    loss, g = train.l2_loss(out, tgt, 4)
    r = out[:, :4] - tgt[:, :4]
    assert loss == pytest.approx(float(np.mean(r * r)), rel=1e-15)
    assert np.all(g[:, 4] == 0.0)
    for idx in [(0, 0, 0, 0), (1, 3, 2, 3), (0, 2, 1, 1), (1, 4, 0, 0)]:
        h = 1e-6
        op, om = out.copy(), out.copy()
        op[idx] += h
        om[idx] -= h
        fd = (train.l2_loss(op, tgt, 4)[0] - train.l2_loss(om, tgt, 4)[0]) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-6, abs=1e-12)
