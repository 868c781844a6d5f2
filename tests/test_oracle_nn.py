"""Pins of the warm-start network oracle against independent implementations:
torch's CPU conv3d, autograd and Adam (library routines), central finite
differences of the oracle's own forward pass, and closed forms."""
import numpy as np
import pytest
import torch

from oracle import nn_oracle as NO
from paper_1809_10895_gb300.workloads import nn_init_params


def _rng(seed=0):
    return np.random.default_rng(seed)


def _torch_net(theta, x):
    """The same network built from torch.nn.functional.conv3d (NCDHW)."""
    layers = NO.unflatten(torch.as_tensor(theta))
    t = torch.as_tensor(x).permute(0, 4, 1, 2, 3)

    def conv(z, W, b):
        return torch.nn.functional.conv3d(z, W.permute(0, 4, 1, 2, 3), b, padding=1)

    a = torch.relu(conv(t, *layers[0]))
    for blk in range(NO.N_BLOCKS):
        u = torch.relu(conv(a, *layers[1 + 2 * blk]))
        a = torch.relu(conv(u, *layers[2 + 2 * blk]) + a)
    return conv(a, *layers[-1])[:, 0]


def test_param_count():
    # 27*4*32+32 + 8*(27*32*32+32) + 27*32+1
    assert NO.n_params() == 3488 + 8 * 27680 + 865


@pytest.mark.parametrize("shape,ci,co", [((1, 5, 4, 3), 4, 6), ((2, 3, 6, 5), 3, 2), ((1, 1, 1, 1), 2, 3)])
def test_conv3d_matches_torch(shape, ci, co):
    rng = _rng(1)
    x = rng.normal(size=shape + (ci,))
    W = rng.normal(size=(co, 3, 3, 3, ci))
    b = rng.normal(size=co)
    ours = NO.conv3d(x, W, b)
    ref = torch.nn.functional.conv3d(torch.as_tensor(x).permute(0, 4, 1, 2, 3),
                                     torch.as_tensor(W).permute(0, 4, 1, 2, 3), torch.as_tensor(b), padding=1)
    np.testing.assert_allclose(ours, ref.permute(0, 2, 3, 4, 1).numpy(), rtol=1e-12, atol=1e-12)


def test_conv3d_single_tap_is_shift():
    # a weight with one non-zero tap is a pure shift with zero fill
    rng = _rng(2)
    x = rng.normal(size=(1, 4, 5, 6, 1))
    W = np.zeros((1, 3, 3, 3, 1))
    W[0, 2, 0, 1, 0] = 1.0          # dz=+1, dy=-1, dx=0
    out = NO.conv3d(x, W, None)[0, ..., 0]
    exp = np.zeros((4, 5, 6))
    exp[:3, 1:, :] = x[0, 1:, :4, :, 0]
    np.testing.assert_array_equal(out, exp)


def test_input_and_weight_grads_match_torch_autograd():
    rng = _rng(3)
    x = rng.normal(size=(1, 4, 3, 5, 3))
    W = rng.normal(size=(2, 3, 3, 3, 3))
    g = rng.normal(size=(1, 4, 3, 5, 2))
    xt = torch.tensor(x, requires_grad=True)
    Wt = torch.tensor(W, requires_grad=True)
    bt = torch.zeros(2, dtype=torch.float64, requires_grad=True)
    out = torch.nn.functional.conv3d(xt.permute(0, 4, 1, 2, 3), Wt.permute(0, 4, 1, 2, 3), bt, padding=1)
    (out.permute(0, 2, 3, 4, 1) * torch.as_tensor(g)).sum().backward()
    np.testing.assert_allclose(NO.conv3d_input_grad(g, W), xt.grad.numpy(), rtol=1e-11, atol=1e-11)
    dW, db = NO.conv3d_weight_grad(x, g)
    np.testing.assert_allclose(dW, Wt.grad.numpy(), rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(db, bt.grad.numpy(), rtol=1e-11, atol=1e-11)


def test_forward_matches_torch_network():
    rng = _rng(4)
    theta = nn_init_params(int(rng.integers(1 << 30))) * 3.0
    x = rng.normal(size=(2, 4, 5, 3, 4))
    y, _, _ = NO.forward(theta, x)
    ref = _torch_net(theta, x).numpy()
    np.testing.assert_allclose(y, ref, rtol=1e-10, atol=1e-12)


def test_gradient_matches_autograd():
    rng = _rng(5)
    theta = nn_init_params(int(rng.integers(1 << 30))) * 3.0
    x = rng.normal(size=(1, 4, 4, 3, 4))
    tgt = rng.normal(size=(1, 4, 4, 3))
    mask = (rng.random((1, 4, 4, 3)) > 0.3).astype(float)
    L, g = NO.loss_and_grad(theta, x, tgt, mask)
    th = torch.tensor(theta, requires_grad=True)
    y = _torch_net(th, x)
    Lt = (((y - torch.as_tensor(tgt)) * torch.as_tensor(mask)) ** 2).sum() / y.numel()
    Lt.backward()
    assert L == pytest.approx(Lt.item(), rel=1e-12)
    np.testing.assert_allclose(g, th.grad.numpy(), rtol=1e-9, atol=1e-13)


def test_gradient_matches_finite_differences():
    rng = _rng(6)
    theta = nn_init_params(int(rng.integers(1 << 30))) * 3.0
    x = rng.normal(size=(1, 3, 3, 3, 4))
    tgt = rng.normal(size=(1, 3, 3, 3))
    _, g = NO.loss_and_grad(theta, x, tgt)
    idx = rng.choice(theta.size, size=40, replace=False)
    idx = np.concatenate([idx, [0, NO.n_params() - 1, 3488 - 1]])   # first weight, last bias, input bias
    for i in idx:
        e = 1e-5 * max(1.0, abs(theta[i]))
        tp, tm = theta.copy(), theta.copy()
        tp[i] += e
        tm[i] -= e
        fd = (NO.loss(NO.forward(tp, x)[0], tgt) - NO.loss(NO.forward(tm, x)[0], tgt)) / (2 * e)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), i


def test_bf16_round_matches_torch():
    rng = _rng(7)
    a = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-20, 20, size=2000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38]])
    ref = torch.as_tensor(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(NO.bf16_round(a), ref)


def test_adam_matches_torch():
    rng = _rng(8)
    w0 = rng.normal(size=50)
    grads = [rng.normal(size=50) for _ in range(4)]
    wt = torch.tensor(w0, requires_grad=True)
    opt = torch.optim.Adam([wt], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    w, m, v = w0.copy(), np.zeros(50), np.zeros(50)
    for t, g in enumerate(grads, start=1):
        w, m, v = NO.adam_step(w, g, m, v, t, lr=3e-3)
        opt.zero_grad()
        wt.grad = torch.as_tensor(g)
        opt.step()
    np.testing.assert_allclose(w, wt.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_bf16_forward_is_close_to_fp64():
    # storage rounding only: |y_bf16 - y| stays a few BF16 ulps of the output scale
    rng = _rng(9)
    theta = nn_init_params(int(rng.integers(1 << 30))) * 3.0
    x = rng.normal(size=(1, 4, 4, 4, 4))
    y = NO.forward(theta, x)[0]
    yb = NO.forward(theta, x, bf16=True)[0]
    assert np.max(np.abs(yb - y)) <= 0.05 * np.max(np.abs(y))


SC = dict(h_scale=2.0, lnK_mean=-11.0, lnK_std=1.5, q_scale=1e-6, t_scale=600.0, out_scale=1e-5)


def test_features_closed_form():
    nz, ny, nx = 3, 2, 2
    h = np.arange(12, dtype=float).reshape(nz, ny, nx) - 6.0
    lnK = np.full((nz, ny, nx), -11.0 + 1.5)
    act = np.ones((nz, ny, nx), bool)
    act[2, 0, 0] = False           # column (0,0) tops out at z index 1
    f = NO.features(h, lnK, act, 2e-6, 60.0, SC)
    assert f[1, 1, 1, 0] == (h[1, 1, 1]) / 2.0
    assert np.all(f[act][:, 1] == 1.0)
    assert f[1, 0, 0, 2] == 2.0 and f[2, 1, 1, 2] == 2.0 and f[1, 1, 1, 2] == 0.0 and f[0, 0, 0, 2] == 0.0
    assert np.allclose(f[act][:, 3], np.log(0.1))
    assert np.all(f[2, 0, 0] == 0.0)


def test_guess_and_target_are_inverse():
    rng = _rng(10)
    h = rng.normal(size=(3, 4, 5))
    h1 = h + 1e-3 * rng.normal(size=h.shape)
    act = rng.random(h.shape) > 0.2
    t = NO.target(h1, h, act, 30.0, SC)
    g = NO.guess(h, t, act, 30.0, SC)
    np.testing.assert_allclose(g[act], h1[act], rtol=0, atol=1e-15)
    np.testing.assert_array_equal(g[~act], h[~act])
