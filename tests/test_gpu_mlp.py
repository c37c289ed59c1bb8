"""GPU parity of the tensor-core deformation MLP (tcgen05 GEMMs) against the
FP64 oracle with the same BF16 operand rounding (oracle/mlp.py).

Layer by layer (tight): each kernel's output is compared with the oracle's
layer applied to the kernel's own inputs (exported from the workspace).  The
oracle sums exactly, the tensor cores in FP32, so an output that lands next to
a BF16 rounding boundary may round the other way: such elements must be rare
(< 1e-3 of a layer) and one BF16 ulp apart, or within the FP32 sum's error
bound (K 2^-24 times the sum of the terms' magnitudes) of zero at the ReLU;
FP32 outputs (head, weight and encoding gradients)
agree to 1e-4 relative.

Against the plain FP64 network (the paper's MLP computes in FP32; BF16
operands are this path's precision choice): offsets within 3u sqrt(9),
u = 2^-8, and gradients within twice the BF16 arithmetic's own distance from
the network (ReLU masks flip near zero) -- test_mlp_against_the_fp64_network.

Whole network (loose, derived): a flipped activation shifts every sum of the
next layer a little and so flips a few more; over 8 layers ~1 % of the
activations end one ulp apart (measured), which moves the output by ~1e-3 and
the deepest weight gradients by ~1e-2 relative -- the difference between two
BF16 evaluations that differ only in summation order.  Bars: output 2e-3,
gradients 2.5e-2 per layer (norm-wise).  The oracle encodes the same
single-precision scaled positions (the top frequency multiplies their
rounding by 2^9 pi)."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_2505_05356_gb300 import gftorf, mlp, scenes

pytestmark = pytest.mark.gpu

ULP = 2.0 ** -7  # one BF16 ulp relative to the value, upper bound


def _case(N, B, seed, head_std=0.05):
    rng = np.random.default_rng(seed)
    theta = scenes.init_mlp_params(seed, head_std=head_std)
    means = rng.uniform(-2.5, 5.0, (N, 3)).astype(np.float32)
    times = list(np.linspace(0.0, 1.0, B).astype(np.float32))
    return theta, means, times


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _bf16_close(got, ref, mag, frac=1e-3):
    """Elementwise equal except rare one-ulp rounding flips, and values
    within the FP32 sum's error bound of zero at the ReLU: a sum of K = 256
    products carries at most K 2^-24 sum|terms| <= 2e-5 mag (mag: the sum of
    the terms' magnitudes, per element)."""
    diff = got != ref
    if not diff.any():
        return True, (0.0,)
    big = np.maximum(np.abs(got), np.abs(ref))[diff]
    d = np.abs(got - ref)[diff]
    ok = (big <= 2e-5 * mag[diff]) | (d <= ULP * big)
    worst = (float(diff.mean()), int((~ok).sum()), float(d[~ok].max()) if (~ok).any() else 0.0)
    return bool(np.all(ok) and diff.mean() <= frac), worst


def _run(N, B, seed):
    theta, means, times = _case(N, B, seed)
    inv = np.float32(1.0 / mlp.unambiguous_range(30e6))
    net = mlp.DeformationMLP(N, B, float(inv))
    th = torch.as_tensor(theta, device="cuda")
    mu = torch.as_tensor(means, device="cuda")
    delta = net.forward(th, mu, times)
    dd = np.random.default_rng(seed + 1).standard_normal((B, N, 3)).astype(np.float32)
    d_theta, d_means = net.backward(th, mu, times, torch.as_tensor(dd, device="cuda"))
    torch.cuda.synchronize()
    net.check()
    return theta, means, times, inv, net, delta, dd, d_theta, d_means


@pytest.mark.parametrize("N,B", [(300, 2), (3000, 3), (77, 1)])
def test_mlp_layer_by_layer(N, B):
    theta, means, times, inv, net, delta, dd, d_theta, d_means = _run(N, B, N + B)
    layers = omlp.unpack(theta.astype(np.float64))
    r = omlp.to_bf16
    # encoding (single-precision scaled positions; sin(pi k) exactly 0 on the GPU)
    enc_g = net.export("enc").double().cpu().numpy()
    enc_o = r(omlp.encode(means, np.asarray(times, np.float64), inv, single=True))
    assert np.abs(enc_g - enc_o).max() <= 1e-6
    H = [net.export("H", l).double().cpu().numpy() for l in range(8)]
    x = enc_g
    for l in range(8):
        W, b = layers[l]
        ref = r(np.maximum(x @ r(W).T + b, 0.0))
        ok, frac = _bf16_close(H[l], ref, np.abs(x) @ np.abs(r(W)).T + np.abs(b))
        assert ok, (l, frac)
        x = H[l]
    Wh, bh = layers[8]
    ref = x @ r(Wh).T + bh
    assert _rel(delta.double().cpu().numpy().reshape(-1, 3), ref) < 1e-5
    # backward, each GEMM from the kernels' own operands
    dZ = [net.export("dZ", l).double().cpu().numpy() for l in range(8)]
    dzh = r(dd.reshape(-1, 3).astype(np.float64))
    ok, frac = _bf16_close(dZ[7], r((dzh @ r(Wh)) * (H[7] > 0)), np.abs(dzh) @ np.abs(r(Wh)))
    assert ok, ("dZ7", frac)
    gt = omlp.unpack(d_theta.double().cpu().numpy())
    assert _rel(gt[8][0], dzh.T @ H[7]) < 1e-4 and _rel(gt[8][1], dzh.sum(0)) < 1e-4
    for l in range(7, -1, -1):
        inp = H[l - 1] if l > 0 else enc_g
        assert _rel(gt[l][0], dZ[l].T @ inp) < 1e-4, ("dW", l)
        assert _rel(gt[l][1], dZ[l].sum(0)) < 1e-4, ("db", l)
        dh = dZ[l] @ r(layers[l][0])
        if l > 0:
            ok, frac = _bf16_close(dZ[l - 1], r(dh * (H[l - 1] > 0)),
                                   np.abs(dZ[l]) @ np.abs(r(layers[l][0])))
            assert ok, ("dZ", l - 1, frac)
        else:
            denc = net.export("d_enc").double().cpu().numpy()
            assert _rel(denc, dh) < 1e-4
            dm = omlp.encode_backward(denc, means, times, inv, single=True)
            assert _rel(d_means.double().cpu().numpy(), dm) < 1e-4


@pytest.mark.parametrize("N,B", [(300, 2), (3000, 3)])
def test_mlp_whole_network_matches_oracle(N, B):
    theta, means, times, inv, net, delta, dd, d_theta, d_means = _run(N, B, 100 + N)
    enc = omlp.encode(means, np.asarray(times, np.float64), inv, single=True)
    d_o, acts = omlp.forward(theta.astype(np.float64), enc, bf16=True)
    g_o, denc = omlp.backward(theta.astype(np.float64), acts, dd.reshape(-1, 3), bf16=True)
    assert _rel(delta.double().cpu().numpy().reshape(-1, 3), d_o) < 2e-3
    for l, ((W, b), (Wo, bo)) in enumerate(zip(omlp.unpack(d_theta.double().cpu().numpy()),
                                              omlp.unpack(g_o))):
        assert _rel(W, Wo) < 2.5e-2 and _rel(b, bo) < 2.5e-2, l
    dm = omlp.encode_backward(denc, means, times, inv, single=True)
    assert _rel(d_means.double().cpu().numpy(), dm) < 2.5e-2


def test_mlp_against_the_fp64_network():
    """The CUDA MLP against the plain FP64 network (Sec. 4: the paper's MLP
    is an FP32 network; this path computes with BF16 operands and FP32
    accumulation).  Bars from BF16's unit roundoff u = 2^-8: each of the 9
    GEMMs rounds its two operands and its output (<= 3u per term; random-sign
    sums keep that relative to the result) and independent layers add in
    quadrature, so the offsets stay within 3u sqrt(9) of the network.  The
    gradients also see ReLU masks that flip where rounding moves a
    pre-activation across zero; such a flip changes a whole dZ element, so
    their distance from the network is the BF16 arithmetic's own (computed
    here by the oracle with BF16 operands, independently of the GPU); the
    CUDA path must stay within twice it, plus the output bar."""
    N, B = 3000, 3
    theta, means, times, inv, net, delta, dd, d_theta, d_means = _run(N, B, 300)
    th64 = theta.astype(np.float64)
    enc = omlp.encode(means, np.asarray(times, np.float64), inv)  # exact scaled positions
    d64, a64 = omlp.forward(th64, enc, bf16=False)
    g64, de64 = omlp.backward(th64, a64, dd.reshape(-1, 3).astype(np.float64), bf16=False)
    d16, a16 = omlp.forward(th64, enc, bf16=True)
    g16, de16 = omlp.backward(th64, a16, dd.reshape(-1, 3).astype(np.float64), bf16=True)
    u = 2.0 ** -8
    out_bar = 3 * u * np.sqrt(9)
    assert _rel(delta.double().cpu().numpy().reshape(-1, 3), d64) <= out_bar
    for l, ((W, b), (W16, b16), (Wo, bo)) in enumerate(
            zip(omlp.unpack(d_theta.double().cpu().numpy()), omlp.unpack(g16),
                omlp.unpack(g64))):
        assert _rel(W, Wo) <= 2 * _rel(W16, Wo) + out_bar, ("W", l, _rel(W, Wo), _rel(W16, Wo))
        assert _rel(b, bo) <= 2 * _rel(b16, bo) + out_bar, ("b", l, _rel(b, bo), _rel(b16, bo))
    dm64 = omlp.encode_backward(de64, means, times, inv)
    dm16 = omlp.encode_backward(de16, means, times, inv)
    dm = d_means.double().cpu().numpy()
    assert _rel(dm, dm64) <= 2 * _rel(dm16, dm64) + out_bar


def test_mlp_zero_gaussians_and_status():
    net = mlp.DeformationMLP(0, 2, 0.2)
    theta = torch.as_tensor(scenes.init_mlp_params(1), device="cuda")
    mu = torch.zeros((0, 3), device="cuda")
    delta = net.forward(theta, mu, [0.0, 1.0])
    d_theta, d_means = net.backward(theta, mu, [0.0, 1.0], torch.zeros((2, 0, 3), device="cuda"))
    torch.cuda.synchronize()
    assert delta.shape == (2, 0, 3) and d_means.shape == (0, 3)
    assert torch.all(d_theta == 0)
    assert net.read_status() == gftorf.OK


def test_mlp_drives_the_renderer_end_to_end():
    """delta from the MLP as the renderer's displacement; the renderer's
    dL/d(delta) back through the MLP; compared with the oracles chained the
    same way."""
    from oracle import oracle as ora
    sc = scenes.make_scene("batch_300k", 21, n=1500, width=64, height=48, frames=2)
    sc.delta = None
    theta = scenes.init_mlp_params(3, head_std=0.02)
    inv = np.float32(1.0 / mlp.unambiguous_range(30e6))
    net = mlp.DeformationMLP(sc.n, sc.frames, float(inv))
    th = torch.as_tensor(theta, device="cuda")
    p = gftorf.params_from_scene(sc)
    times = [float(t) for t in sc.times]
    p["delta"] = net.forward(th, p["means"], times)
    r = gftorf.Renderer(sc.n, sc.frames, sc.width, sc.height, 1, 4)
    fr, se, co = (gftorf.frames_from_scene(sc), gftorf.sensor_from_scene(sc),
                  gftorf.consts_from_scene(sc))
    bg = torch.as_tensor(sc.bg, device="cuda")
    r.fit_capacity(p, fr, se, co, bg)
    r.preprocess(p, fr, se, co)
    out = r.render_fwd(bg)
    # the oracle renders with the GPU's delta (its own MLP is checked above)
    sc.delta = p["delta"].double().cpu().numpy()
    q_o, _, amb, _ = ora.render(sc, ora.EPS_F32)
    keep = (amb & ora.AMB_VALUE) == 0
    err = np.abs(out.double().cpu().numpy() - q_o).transpose(1, 0, 2, 3)[:, keep]
    assert err.max() <= 1e-5 * np.abs(q_o).max()
    dout = scenes.random_dout(sc, 5)
    dout[np.broadcast_to((amb != 0)[:, None], dout.shape)] = 0.0
    g = r.render_bwd(p, bg, torch.as_tensor(dout, device="cuda"))
    d_theta, d_means = net.backward(th, p["means"], times, g["delta"])
    torch.cuda.synchronize()
    go = ora.backward(sc, dout.astype(np.float64))
    assert _rel(g["delta"].double().cpu().numpy(), go["delta"]) < 1e-3
    # the MLP backward from the oracle's dL/d(delta) through the oracle MLP
    enc = omlp.encode(sc.means, np.asarray(times), inv, single=True)
    _, acts = omlp.forward(theta.astype(np.float64), enc, bf16=True)
    g_th, denc = omlp.backward(theta.astype(np.float64), acts, go["delta"].reshape(-1, 3),
                               bf16=True)
    assert _rel(d_theta.double().cpu().numpy(), g_th) < 2.5e-2
    dm_o = omlp.encode_backward(denc, sc.means, times, inv, single=True) + go["means"]
    assert _rel(d_means.double().cpu().numpy() + g["means"].double().cpu().numpy(), dm_o) < 2.5e-2


def test_bounded_waits_report_timeout_and_leave_the_context_usable():
    """With the load warps told to issue nothing, every GEMM's waits run out
    (50 ms each under injection): the status word reports the timeout, the
    kernels return, and the next call on the same context is correct."""
    N, B = 100, 1
    theta, means, times = _case(N, B, 41)
    inv = np.float32(0.2)
    net = mlp.DeformationMLP(N, B, float(inv))
    th = torch.as_tensor(theta, device="cuda")
    mu = torch.as_tensor(means, device="cuda")
    mlp.debug_inject(1)
    try:
        net.forward(th, mu, times)
        assert net.read_status() == gftorf.ERR_TIMEOUT
    finally:
        mlp.debug_inject(0)
    delta = net.forward(th, mu, times)
    assert net.read_status() == gftorf.OK
    enc = omlp.encode(means, np.asarray(times, np.float64), inv, single=True)
    d_o, _ = omlp.forward(theta.astype(np.float64), enc, bf16=True)
    assert _rel(delta.double().cpu().numpy().reshape(-1, 3), d_o) < 2e-3


@pytest.mark.parametrize("N,B", [(300, 2), (3000, 3), (77, 1), (40000, 2)])
def test_fused_inference_equals_layer_by_layer_forward(N, B):
    """The fused kernel (activations in shared memory) performs the same
    arithmetic in the same order: bit-identical offsets."""
    theta, means, times = _case(N, B, 50 + N)
    net = mlp.DeformationMLP(N, B, 0.2)
    th = torch.as_tensor(theta, device="cuda")
    mu = torch.as_tensor(means, device="cuda")
    mlp.debug_inject(2)  # the reference: one GEMM per layer
    try:
        ref = net.forward(th, mu, times).clone()
    finally:
        mlp.debug_inject(0)
    got = net.infer(th, mu, times)
    torch.cuda.synchronize()
    assert net.read_status() == gftorf.OK
    np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())


@pytest.mark.parametrize("N,B", [(300, 2), (3000, 3), (77, 1), (40000, 2)])
def test_fused_training_forward_keeps_what_the_layerwise_one_keeps(N, B):
    """The fused training forward stores the same transposed activations,
    encoding and ReLU masks as the one-GEMM-per-layer forward, and the fused
    backward chain forms the same dZ of every layer and the same encoding
    gradient (same operands, same MMA order): bit-identical.  (40000, 2):
    more tile pairs than SMs, so CTAs loop; (77, 1): one ragged tile.)"""
    theta, means, times = _case(N, B, 60 + N)
    net = mlp.DeformationMLP(N, B, 0.2)
    th = torch.as_tensor(theta, device="cuda")
    mu = torch.as_tensor(means, device="cuda")
    dd = torch.as_tensor(np.random.default_rng(4).standard_normal((B, N, 3)).astype(np.float32),
                         device="cuda")

    def run():
        d = net.forward(th, mu, times).clone()
        keep = [net.export("enc").clone()] + [net.export("H", l).clone() for l in range(8)]
        g, m = net.backward(th, mu, times, dd)
        dz = [net.export("dZ", l).clone() for l in range(8)] + [net.export("d_enc").clone()]
        torch.cuda.synchronize()
        return d, keep, g.clone(), m.clone(), dz

    mlp.debug_inject(2)
    try:
        ref = run()
    finally:
        mlp.debug_inject(0)
    got = run()
    assert net.read_status() == gftorf.OK
    np.testing.assert_array_equal(got[0].cpu().numpy(), ref[0].cpu().numpy())
    for a, b in zip(got[1], ref[1]):
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
    for a, b in zip(got[4], ref[4]):
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
    # hidden weight gradients: the same GEMM on the same operands, reduced in
    # a fixed order -- equal; the biases (column sums) and the head's weights
    # sum with atomics: equal up to summation order, i.e. within an FP32
    # summation bound of 64 ulp of the sum of the terms' magnitudes (the terms
    # cancel: the sums are ~1 % of their magnitudes at these sizes)
    bound = 64 * 2.0 ** -24
    dzs = [z.double().cpu().numpy() for z in got[4][:8]]
    ddh = np.abs(dd.double().cpu().numpy().reshape(-1, 3))
    h7 = np.abs(got[1][8].double().cpu().numpy())
    gl = omlp.unpack(got[2].double().cpu().numpy())
    rl = omlp.unpack(ref[2].double().cpu().numpy())
    for l in range(8):
        np.testing.assert_array_equal(gl[l][0], rl[l][0])
        mag = np.abs(dzs[l]).sum(0)
        assert np.all(np.abs(gl[l][1] - rl[l][1]) <= bound * mag), l
    assert np.all(np.abs(gl[8][0] - rl[8][0]) <= bound * (ddh.T @ h7))
    assert np.all(np.abs(gl[8][1] - rl[8][1]) <= bound * ddh.sum(0))
    np.testing.assert_array_equal(got[3].cpu().numpy(), ref[3].cpu().numpy())


def test_fused_backward_bounded_waits():
    """The fused backward's waits run out under injection: timeout in the
    status word, the context stays usable, and the next backward matches."""
    N, B = 100, 1
    theta, means, times = _case(N, B, 45)
    net = mlp.DeformationMLP(N, B, 0.2)
    th = torch.as_tensor(theta, device="cuda")
    mu = torch.as_tensor(means, device="cuda")
    dd = torch.as_tensor(np.random.default_rng(5).standard_normal((B, N, 3)).astype(np.float32),
                         device="cuda")
    net.forward(th, mu, times)
    g_ref, m_ref = (t.clone() for t in net.backward(th, mu, times, dd))
    assert net.read_status() == gftorf.OK
    mlp.debug_inject(1)
    try:
        net.backward(th, mu, times, dd)
        assert net.read_status() == gftorf.ERR_TIMEOUT
    finally:
        mlp.debug_inject(0)
    net.forward(th, mu, times)
    g, m = net.backward(th, mu, times, dd)
    assert net.read_status() == gftorf.OK
    assert _rel(g.double().cpu().numpy(), g_ref.double().cpu().numpy()) < 1e-6
    np.testing.assert_array_equal(m.cpu().numpy(), m_ref.cpu().numpy())


def test_fused_inference_bounded_waits():
    N, B = 100, 1
    theta, means, times = _case(N, B, 43)
    net = mlp.DeformationMLP(N, B, 0.2)
    th = torch.as_tensor(theta, device="cuda")
    mu = torch.as_tensor(means, device="cuda")
    mlp.debug_inject(1)
    try:
        net.infer(th, mu, times)
        assert net.read_status() == gftorf.ERR_TIMEOUT
    finally:
        mlp.debug_inject(0)
    ref = net.forward(th, mu, times).clone()
    got = net.infer(th, mu, times)
    assert net.read_status() == gftorf.OK
    np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())
