"""Pins of the deformation-MLP oracle (oracle/mlp.py): the positional
encoding's closed form, the network and its hand-written backward against
torch's float64 layers and autograd (a library routine), central differences,
and the bfloat16 rounding against torch's conversion."""
import math

import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2505_05356_gb300 import scenes

torch = pytest.importorskip("torch")


def _theta(seed, head_std=0.05):
    return scenes.init_mlp_params(seed, head_std=head_std).astype(np.float64)


def test_encoding_closed_form():
    du = 5.0
    enc = omlp.encode([[0.25 * du, 0.5 * du, 0.0]], [0.5], 1.0 / du)
    assert enc.shape == (1, 128)
    e = enc[0]
    np.testing.assert_allclose(e[0:3], [0.25, 0.5, 0.0], atol=1e-15)
    # l = 0: sin(pi x), cos(pi x); l = 1: sin(2 pi x), cos(2 pi x)
    np.testing.assert_allclose(e[3:6], [math.sqrt(0.5), 1.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(e[6:9], [math.sqrt(0.5), 0.0, 1.0], atol=1e-15)
    np.testing.assert_allclose(e[9:12], [1.0, 0.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(e[12:15], [0.0, -1.0, 1.0], atol=1e-15)
    # time block: t, sin(pi t) = 1, cos(pi t) = 0, sin(2 pi t) = 0, cos(2 pi t) = -1
    np.testing.assert_allclose(e[63:68], [0.5, 1.0, 0.0, 0.0, -1.0], atol=1e-15)
    assert np.all(e[84:] == 0.0)


def _torch_net(theta, enc):
    layers = omlp.unpack(theta)
    h = torch.tensor(enc, dtype=torch.float64, requires_grad=True)
    params = [(torch.tensor(W, requires_grad=True), torch.tensor(b, requires_grad=True))
              for W, b in layers]
    x = h
    for W, b in params[:-1]:
        x = torch.relu(torch.nn.functional.linear(x, W, b))
    out = torch.nn.functional.linear(x, *params[-1])
    return h, params, out


def test_forward_and_backward_match_torch_fp64():
    rng = np.random.default_rng(1)
    theta = _theta(2)
    enc = omlp.encode(rng.uniform(0, 5, (7, 3)), [0.1, 0.6], 0.2)
    delta, acts = omlp.forward(theta, enc, bf16=False)
    h, params, out = _torch_net(theta, enc)
    np.testing.assert_allclose(delta, out.detach().numpy(), rtol=1e-12, atol=1e-15)
    g = rng.standard_normal(delta.shape)
    d_theta, d_enc = omlp.backward(theta, acts, g, bf16=False)
    (out * torch.tensor(g)).sum().backward()
    ref = np.concatenate([np.concatenate([W.grad.numpy().reshape(-1), b.grad.numpy()])
                          for W, b in params])
    np.testing.assert_allclose(d_theta, ref, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(d_enc, h.grad.numpy(), rtol=1e-10, atol=1e-14)


def test_backward_central_differences():
    rng = np.random.default_rng(3)
    theta = _theta(4)
    enc = omlp.encode(rng.uniform(0, 5, (5, 3)), [0.3], 0.2)
    g = rng.standard_normal((5, 3))
    d_theta, _ = omlp.backward(theta, omlp.forward(theta, enc, bf16=False)[1], g, bf16=False)
    L = lambda th: float(np.sum(omlp.forward(th, enc, bf16=False)[0] * g))
    nz = np.flatnonzero(d_theta)
    for i in rng.choice(nz, 40, replace=False):
        h = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (L(tp) - L(tm)) / (2 * h)
        assert d_theta[i] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_encode_backward_central_differences():
    rng = np.random.default_rng(5)
    means = rng.uniform(0, 5, (4, 3))
    times = [0.2, 0.7, 0.9]
    d_enc = rng.standard_normal((12, 128))
    d_enc[:, 84:] = 0.0
    g = omlp.encode_backward(d_enc, means, times, 0.2)
    for gi in range(4):
        for a in range(3):
            h = 1e-6
            mp, mm = means.copy(), means.copy()
            mp[gi, a] += h
            mm[gi, a] -= h
            fd = (np.sum(d_enc * omlp.encode(mp, times, 0.2)) -
                  np.sum(d_enc * omlp.encode(mm, times, 0.2))) / (2 * h)
            assert g[gi, a] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(6)
    x = np.concatenate([rng.standard_normal(1000) * 10.0 ** rng.integers(-8, 8, 1000),
                        [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 0.0]])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(omlp.to_bf16(x), ref)


def test_bf16_network_close_to_fp64():
    rng = np.random.default_rng(7)
    theta = _theta(8, head_std=0.05)
    enc = omlp.encode(rng.uniform(0, 5, (64, 3)), [0.5], 0.2)
    d64, _ = omlp.forward(theta, enc, bf16=False)
    d16, _ = omlp.forward(theta, enc, bf16=True)
    assert np.linalg.norm(d16 - d64) / np.linalg.norm(d64) < 3e-2
