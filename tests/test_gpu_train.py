"""GPU parity of the optimisation-loop steps against the FP64 oracle
(oracle/train.py): the random background (bit-exact), the raw-sample L2 loss
and its gradient, the fused projected Adam, one whole fitting iteration, and
the same iteration replayed from a CUDA graph."""
import numpy as np
import pytest
import torch

from oracle import oracle as ora
from oracle import train as otrain
from paper_2505_05356_gb300 import fit, gftorf, scenes
from tests.gpu_helpers import grads_close

pytestmark = pytest.mark.gpu


def test_background_stream_bit_exact():
    st = gftorf.new_train_state()
    bg = torch.empty((3, 7), device="cuda")
    seen = []
    for _ in range(4):
        gftorf.train_begin(st, bg, seed=1234)
        seen.append(bg.cpu().numpy().astype(np.float64))
    ref = otrain.background_sample(1234, 4, 21)
    np.testing.assert_array_equal(np.stack(seen).reshape(4, 21), ref)
    assert gftorf.train_step_count(st) == 4 and gftorf.train_loss(st) == 0.0


@pytest.mark.parametrize("W,H,extra", [(50, 37, False), (64, 48, False), (64, 48, True)])
def test_l2_loss_matches_oracle(W, H, extra):
    sc = scenes.make_scene("batch_300k", 3, n=10, width=W, height=H, frames=3,
                           freqs_hz=[30e6, 80e6], phasor=extra, depth=extra)
    r = gftorf.Renderer(sc.n, sc.frames, W, H, 2, 4, flags=gftorf.flags_from_scene(sc))
    rng = np.random.default_rng(5)
    out = rng.standard_normal((sc.frames, r.C, H, W)).astype(np.float32)
    tgt = rng.standard_normal((sc.frames, r.C, H, W)).astype(np.float32)
    st = gftorf.new_train_state()
    gftorf.train_begin(st, None, 0)
    dout = torch.full((sc.frames, r.C, H, W), 7.0, device="cuda")
    gftorf.l2_loss(r, torch.as_tensor(out, device="cuda"), torch.as_tensor(tgt, device="cuda"),
                   dout, st)
    loss_o, g_o = otrain.l2_loss(out, tgt, 8)
    assert gftorf.train_loss(st) == pytest.approx(loss_o, rel=1e-5)
    np.testing.assert_allclose(dout.cpu().numpy(), g_o, rtol=1e-6, atol=1e-12)


def test_adam_matches_oracle_over_steps():
    rng = np.random.default_rng(9)
    shapes = {"a": (1000, 3), "b": (777,), "c": (5, 4, 3)}
    lrs = {"a": 1e-3, "b": 5e-2, "c": 1.6e-4}
    bounds = {"b": (1e-4, 1.0)}
    p_np = {k: rng.uniform(0.01, 1.0, s).astype(np.float32) for k, s in shapes.items()}
    params = {k: torch.as_tensor(v, device="cuda") for k, v in p_np.items()}
    opt = gftorf.Adam(params, lrs, bounds)
    st = gftorf.new_train_state()
    ref = {k: (v.astype(np.float64), 0.0, 0.0) for k, v in p_np.items()}
    for t in range(1, 5):
        g_np = {k: (rng.standard_normal(s) * 10.0 ** rng.integers(-6, 1)).astype(np.float32)
                for k, s in shapes.items()}
        gftorf.train_begin(st, None, 0)
        opt.step({k: torch.as_tensor(v, device="cuda") for k, v in g_np.items()}, st)
        for k in shapes:
            p, m, v = ref[k]
            lo, hi = bounds.get(k, (-np.inf, np.inf))
            # the oracle steps from the GPU's current value (float32), so the
            # comparison is per step, not compounded
            p_prev = p
            ref[k] = otrain.adam_step(p_prev, g_np[k].astype(np.float64), m, v, t, lrs[k],
                                      lo=lo, hi=hi)
            got = params[k].cpu().numpy().astype(np.float64)
            np.testing.assert_allclose(got, ref[k][0], rtol=2e-6, atol=2e-5 * lrs[k] * t)
            ref[k] = (got, ref[k][1], ref[k][2])
        assert np.all(params["b"].cpu().numpy() >= 1e-4)


FIT_LRS = fit.LEARNING_RATES
FIT_BOUNDS = fit.BOUNDS


def _same_fit(pa, pb, steps):
    """Two fits of the same steps whose gradients differ only in atomic
    summation order: Adam's early steps move each parameter by about
    lr sign(g), so an element whose gradient sums to nearly zero may step the
    other way -- rare, and at most 2 lr per step; all others agree closely."""
    for k, lr in FIT_LRS.items():
        a, b = pa[k].double().cpu().numpy(), pb[k].double().cpu().numpy()
        close = np.isclose(a, b, rtol=1e-4, atol=1e-4 * lr)
        assert close.mean() >= 1 - 1e-3, (k, float(close.mean()))
        assert np.all(np.abs(a - b) <= 2 * steps * lr * (1 + 1e-3) + 1e-4 * np.abs(b)), k


def _fit_setup(seed=4, n=2500, frames=4, W=64, H=48):
    gt, init = scenes.make_fit_scenes(seed, n_backdrop=int(0.9 * n), n_rod=n - int(0.9 * n),
                                      n_init=n, frames=frames, width=W, height=H)
    target = ora.render(gt)[0].astype(np.float32)  # targets from the oracle
    return gt, init, target


def test_one_fitting_iteration_matches_oracle():
    gt, init, target = _fit_setup()
    B, W, H = init.frames, init.width, init.height
    r = gftorf.Renderer(init.n, B, W, H, 1, 4)
    p = gftorf.params_from_scene(init)
    fr, se, co = (gftorf.frames_from_scene(init), gftorf.sensor_from_scene(init),
                  gftorf.consts_from_scene(init))
    bg = torch.empty((B, r.C), device="cuda")
    st = gftorf.new_train_state()
    r.fit_capacity(p, fr, se, co, torch.zeros((B, r.C), device="cuda"))
    tgt = torch.as_tensor(target, device="cuda")
    out = torch.empty((B, r.C, H, W), device="cuda")
    dout = torch.empty_like(out)
    opt = gftorf.Adam(p, FIT_LRS, FIT_BOUNDS)
    before = {k: v.clone() for k, v in p.items() if v is not None}
    gftorf.train_begin(st, bg, seed=77)
    r.preprocess(p, fr, se, co)
    r.render_fwd(bg, out)
    gftorf.l2_loss(r, out, tgt, dout, st)
    grads = r.render_bwd(p, bg, dout, want=list(FIT_LRS))
    g_gpu = {k: v.double().cpu().numpy() for k, v in grads.items()}
    opt.step(grads, st)
    torch.cuda.synchronize()
    # oracle: same background, loss, gradient and update
    bg_o = otrain.background_sample(77, 1, B * r.C).reshape(B, r.C)
    np.testing.assert_array_equal(bg.cpu().numpy(), bg_o)
    init.bg = bg_o
    q_o, _, amb, _ = ora.render(init, ora.EPS_F32)
    loss_o, dq_o = otrain.l2_loss(q_o, target, 4)
    assert gftorf.train_loss(st) == pytest.approx(loss_o, rel=1e-4)
    dq_o[np.broadcast_to((amb != 0)[:, None], dq_o.shape)] = 0.0
    g_o = ora.backward(init, dq_o)
    errs = grads_close(g_gpu, g_o, rel=1e-3, absent=set(g_o) - set(FIT_LRS))
    # ambiguous pixels were zeroed only on the oracle side: compare norm-wise
    for k, (nrm, elem) in errs.items():
        assert nrm <= 5e-3, (k, nrm)
    # the update applied to the GPU's own gradients equals the oracle's Adam
    for k, lr in FIT_LRS.items():
        lo, hi = FIT_BOUNDS.get(k, (-np.inf, np.inf))
        exp, _, _ = otrain.adam_step(before[k].double().cpu().numpy(), g_gpu[k], 0.0, 0.0, 1,
                                     lr, lo=lo, hi=hi)
        np.testing.assert_allclose(p[k].double().cpu().numpy(), exp, rtol=2e-6,
                                   atol=2e-5 * lr)


def test_graph_replayed_iterations_equal_eager_ones():
    gt, init, target = _fit_setup(seed=6)

    def make():
        p = gftorf.params_from_scene(init)
        return fit.FitLoop(p, gftorf.frames_from_scene(init), gftorf.sensor_from_scene(init),
                           gftorf.consts_from_scene(init), torch.as_tensor(target, device="cuda"),
                           tile=(16, 32), pixels_per_thread=4, render_mode=1, seed=5,
                           headroom=2.0), p

    eager, p1 = make()
    eager.run(3)
    graphed, p2 = make()
    graphed.capture()
    # capturing does not run the work: the state is still at step 0
    assert graphed.step == 0
    graphed.run(3)
    torch.cuda.synchronize()
    assert eager.step == graphed.step == 3
    eager.check()
    graphed.check()
    assert graphed.loss() == pytest.approx(eager.loss(), rel=1e-5)
    _same_fit(p2, p1, 3)

def test_fit_reduces_the_loss():
    """With the background held at 0 (so the loss is not redrawn every
    iteration) the fitted parameters move downhill."""
    gt, init, target = _fit_setup(seed=8)
    p = gftorf.params_from_scene(init)
    loop = fit.FitLoop(p, gftorf.frames_from_scene(init), gftorf.sensor_from_scene(init),
                       gftorf.consts_from_scene(init), torch.as_tensor(target, device="cuda"),
                       random_background=False, headroom=2.0)
    loop.capture()
    loop.run(1)
    first = loop.loss()
    loop.run(30)
    loop.check()
    assert loop.loss() < 0.98 * first


def test_checkpoint_resume_continues_the_same_fit(tmp_path):
    """A fit checkpointed after 3 iterations and resumed in a fresh loop (from
    the file) draws the same next background and renders a bit-identical
    forward in the next iteration."""
    gt, init, target = _fit_setup(seed=9)

    def make():
        p = gftorf.params_from_scene(init)
        return fit.FitLoop(p, gftorf.frames_from_scene(init), gftorf.sensor_from_scene(init),
                           gftorf.consts_from_scene(init), torch.as_tensor(target, device="cuda"),
                           seed=13, headroom=2.0)

    a = make()
    a.run(3)
    path = tmp_path / "fit.pt"
    torch.save(a.state_dict(), path)
    a.run(1)
    torch.cuda.synchronize()
    b = make()
    b.capture()  # resume into a captured loop: the graph's buffers are reused
    b.load_state_dict(torch.load(path))
    assert b.step == 3
    b.run(1)
    torch.cuda.synchronize()
    assert b.step == a.step == 4
    np.testing.assert_array_equal(b.bg.cpu().numpy(), a.bg.cpu().numpy())
    np.testing.assert_array_equal(b.out.cpu().numpy(), a.out.cpu().numpy())
    a.check()
    b.check()


def test_background_shards_are_slices_of_the_batch_draw():
    """A shard of frames draws exactly its slice of the whole batch's
    background stream, every iteration (bit for bit, against the oracle's
    stream of the whole batch)."""
    B, C, seed = 6, 5, 99
    full = otrain.background_sample(seed, 3, B * C).reshape(3, B, C)
    for a, b in ((0, 2), (2, 5), (5, 6)):
        st = gftorf.new_train_state()
        bg = torch.empty((b - a, C), device="cuda")
        for s in range(3):
            gftorf.train_begin(st, bg, seed, bg_offset=a * C, bg_stride=B * C)
            np.testing.assert_array_equal(bg.cpu().numpy().astype(np.float64), full[s, a:b])


def test_frame_shards_add_up_to_the_whole_batch():
    """One fitting iteration of a 4-frame batch run as two 2-frame shards (one
    after the other on this GPU, as two processes would run them): the
    shards' background slices, losses and parameter gradients add up to the
    whole batch's, and after the gradient sum (the all-reduce of a sharded
    fit) both shards take the same Adam step."""
    gt, init, target = _fit_setup(seed=9)
    B = init.frames
    fr, se, co = (gftorf.frames_from_scene(init), gftorf.sensor_from_scene(init),
                  gftorf.consts_from_scene(init))
    tgt = torch.as_tensor(target, device="cuda")

    def loop(a, b):
        p = gftorf.params_from_scene(init)
        return fit.FitLoop(p, fr[a:b], se, co, tgt[a:b].contiguous(), seed=13, headroom=2.0,
                           frame_offset=a, total_frames=B), p

    whole, pw = loop(0, B)
    parts = [loop(0, 2), loop(2, B)]
    whole.forward_backward()
    for lp, _ in parts:
        lp.forward_backward()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(torch.cat([lp.bg for lp, _ in parts]).cpu().numpy(),
                                  whole.bg.cpu().numpy())
    assert sum(lp.loss() for lp, _ in parts) == pytest.approx(whole.loss(), rel=1e-6)
    gsum = {k: sum(lp.param_grads()[k] for lp, _ in parts) for k in whole.param_grads()}
    for k, g in whole.param_grads().items():
        ref = g.double().cpu().numpy()
        got = gsum[k].double().cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref), k
    for lp, _ in parts:  # the all-reduce's result on every process
        for k, g in lp.param_grads().items():
            g.copy_(gsum[k])
        lp.update()
    torch.cuda.synchronize()
    for k in FIT_LRS:
        np.testing.assert_array_equal(parts[0][1][k].cpu().numpy(), parts[1][1][k].cpu().numpy())


def test_grad_hook_runs_between_two_graphs():
    """With a grad_hook the iteration is captured as two graphs with the hook
    between their replays; an identity hook leaves the fit as without one."""
    gt, init, target = _fit_setup(seed=10)

    def make(hook):
        p = gftorf.params_from_scene(init)
        return fit.FitLoop(p, gftorf.frames_from_scene(init), gftorf.sensor_from_scene(init),
                           gftorf.consts_from_scene(init), torch.as_tensor(target, device="cuda"),
                           seed=3, headroom=2.0, grad_hook=hook), p

    calls = []
    hooked, p1 = make(lambda g: calls.append(sorted(g)))
    hooked.capture()
    hooked.run(3)
    plain, p2 = make(None)
    plain.capture()
    plain.run(3)
    torch.cuda.synchronize()
    assert len(calls) == 3 and calls[0] == sorted(FIT_LRS)
    assert hooked.step == plain.step == 3
    assert hooked.loss() == pytest.approx(plain.loss(), rel=1e-5)
    _same_fit(p1, p2, 3)
