"""The warm-start network's BF16 kernels against the FP64 reference (oracle/mlp.py), which
rounds to BF16 at the points where the kernels store BF16: forward output, gradients of
every parameter, the fitted normalisation, one Adam step, and training on a regression."""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu

SIZES = [32, 256, 256, 256, 7]


@pytest.fixture(scope="module")
def ws():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2302_14344_gb300 import warmstart
    return warmstart


def _setup(ws, seed=0, B=300):
    import torch
    rng = np.random.default_rng(seed)
    params = mlp.init_params(SIZES, seed=seed)
    params = [(W.astype(np.float32).astype(np.float64),
               (rng.standard_normal(b.shape) * 0.1).astype(np.float32).astype(np.float64))
              for W, b in params]
    x = rng.standard_normal((B, SIZES[0])).astype(np.float32)
    t = rng.standard_normal((B, SIZES[-1])).astype(np.float32)
    mask = (rng.random((B, SIZES[-1])) < 0.85).astype(np.float32)
    net = ws.Network(SIZES)
    net.set_params(ws.join_params(params))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return net, params, x, t, mask, dev


def _rel(a, b):
    return np.linalg.norm(np.asarray(a, float) - b) / max(np.linalg.norm(b), 1e-30)


def test_forward_matches_the_bf16_reference(ws):
    import torch
    net, params, x, t, mask, dev = _setup(ws)
    y = torch.empty((x.shape[0], SIZES[-1]), device="cuda")
    net.forward(dev(x), y)
    ref, _ = mlp.forward(params, x.astype(np.float64), bf16=True)
    assert _rel(y.cpu().numpy(), ref) < 2e-3


def test_gradients_match_the_bf16_reference(ws, capsys):
    import torch
    net, params, x, t, mask, dev = _setup(ws, seed=1)
    grad = torch.zeros(net.num_params, device="cuda")
    loss = torch.zeros(1, device="cuda")
    net.gradients(dev(x), dev(t), dev(mask), grad, loss)
    y, cache = mlp.forward(params, x.astype(np.float64), bf16=True)
    ref = mlp.backward(params, cache, y, t.astype(np.float64), mask.astype(np.float64), bf16=True)
    got = ws.split_params(grad.cpu().numpy().astype(np.float64), SIZES)
    worst = 0.0
    for (gw, gb), (rw, rb) in zip(got, ref):
        worst = max(worst, _rel(gw, rw), _rel(gb, rb))
    with capsys.disabled():
        print(f"\n[BF16 network gradients vs FP64 reference (BF16-rounded storage)] worst "
              f"relative error over parameter arrays {worst:.2e}")
    assert worst < 5e-3
    assert np.isclose(loss.item(), mlp.loss(y, t.astype(np.float64), mask), rtol=1e-3)


def test_fitted_normalization_is_mean_std_and_rms(ws):
    import torch
    net, params, x, t, mask, dev = _setup(ws, seed=2, B=5000)
    x = x * np.linspace(0.5, 3.0, SIZES[0]).astype(np.float32) + 2.0
    x[:, 5] = 7.0                                   # a constant column keeps std 1
    net.fit_normalization(dev(x), dev(t))
    m, s, o = net.get_normalization()
    xs = x.astype(np.float64)
    sd = xs.std(axis=0)
    sd[5] = 1.0
    assert np.allclose(m, xs.mean(axis=0), rtol=1e-5, atol=1e-5)
    assert np.allclose(s, sd, rtol=1e-4)
    assert np.allclose(o, np.sqrt((t.astype(np.float64) ** 2).mean(axis=0)), rtol=1e-5)


def test_one_adam_step_matches_the_reference_step_on_the_same_gradients(ws):
    import torch
    net, params, x, t, mask, dev = _setup(ws, seed=3)
    grad = torch.zeros(net.num_params, device="cuda")
    net.gradients(dev(x), dev(t), dev(mask), grad)
    g = ws.split_params(grad.cpu().numpy().astype(np.float64), SIZES)
    net.train_step(dev(x), dev(t), dev(mask), 1e-3)
    after = ws.split_params(net.get_params().astype(np.float64), SIZES)
    ref = [(W.copy(), b.copy()) for W, b in params]
    mlp.adam(ref, g, [], lr=1e-3, t=1)
    for (aw, ab), (rw, rb) in zip(after, ref):
        assert np.abs(aw - rw).max() < 2e-6 and np.abs(ab - rb).max() < 2e-6


def test_training_reduces_the_loss_of_a_smooth_regression(ws, capsys):
    import torch
    rng = np.random.default_rng(4)
    B = 4096
    x = rng.standard_normal((B, SIZES[0])).astype(np.float32)
    A = rng.standard_normal((SIZES[0], SIZES[-1])) / np.sqrt(SIZES[0])
    t = (np.tanh(x @ A) + 0.1 * (x[:, :SIZES[-1]] ** 2)).astype(np.float32)
    mask = np.ones_like(t)
    net = ws.Network(SIZES)
    net.set_params(ws.join_params(mlp.init_params(SIZES, seed=4)))
    xd, td, md = (torch.from_numpy(a).cuda() for a in (x, t, mask))
    net.fit_normalization(xd, td)
    losses = []
    for it in range(300):
        loss = torch.zeros(1, device="cuda")
        lo = (it * 512) % B
        net.train_step(xd[lo:lo + 512].contiguous(), td[lo:lo + 512].contiguous(),
                       md[lo:lo + 512].contiguous(), 1e-3, loss)
        losses.append(loss.item())
    with capsys.disabled():
        print(f"\n[warm-start network training, smooth regression] loss {losses[0]:.3e} -> "
              f"{np.mean(losses[-10:]):.3e}")
    assert np.mean(losses[-10:]) < 0.1 * losses[0]


@pytest.mark.parametrize("B", [1, 127, 128, 129, 1000, 70001])
def test_fused_tensor_core_forward_equals_the_layered_forward(ws, B):
    """All four layers in one tcgen05 launch (tiles of 128 interfaces, ragged last tile)
    against the layer-by-layer kernels, with a fitted input normalisation and output scale:
    the same BF16/FP32 arithmetic, so they agree to the order of the FP32 sums (an
    activation may round to the neighbouring BF16 value)."""
    import torch
    net, params, _, _, _, dev = _setup(ws, seed=4, B=8)
    g = torch.Generator(device="cuda").manual_seed(B)
    x = torch.randn(B, SIZES[0], device="cuda", generator=g) * 3.0 + 1.0
    t = torch.randn(B, SIZES[-1], device="cuda", generator=g) * 5.0
    net.fit_normalization(x, t)
    y = torch.full((B, SIZES[-1]), float("nan"), device="cuda")
    z = torch.empty((B, SIZES[-1]), device="cuda")
    net.forward(x, y)
    net.forward_layers(x, z)
    torch.cuda.synchronize()
    assert net.fused_error() == 0
    assert torch.isfinite(y).all()
    err = float((y - z).norm() / z.norm())
    assert err < 3e-3, err


def test_fused_forward_follows_training(ws):
    """The fused path packs the current BF16 weights on every call: after Adam steps its
    outputs follow the layer-by-layer path's."""
    import torch
    net, params, x, t, mask, dev = _setup(ws, seed=6)
    for _ in range(3):
        net.train_step(dev(x), dev(t), dev(mask), 1e-2)
    y = torch.empty((x.shape[0], SIZES[-1]), device="cuda")
    z = torch.empty_like(y)
    net.forward(dev(x), y)
    net.forward_layers(dev(x), z)
    torch.cuda.synchronize()
    assert float((y - z).norm() / z.norm()) < 3e-3
