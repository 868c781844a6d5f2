"""Warm-start network on the GPU against the FP64 network oracle, through
the C ABI: forward pass, loss gradient, Adam step, solver features and
targets; warm-started steps against the plain oracle; the fallback; and what
a network trained by these kernels gains over the method without it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import nn_oracle as NO
from paper_1809_10895_gb300 import rf, warmstart
from paper_1809_10895_gb300 import workloads as W
from tests.helpers import oracle_from_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1809_10895_gb300 import build as B
    B.build()
    rf.load()
    torch.cuda.set_device(0)


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def theta_f32(seed, scale=3.0):
    # parameters exchanged as FP32: the oracle takes the same rounded values
    return (W.nn_init_params(seed) * scale).astype(np.float32).astype(np.float64)


# Volumes spanning several 128-voxel conv tiles with ragged tails, one voxel,
# and a batch of two.
SHAPES = [(1, 5, 7, 9), (2, 3, 6, 11), (1, 1, 1, 1), (1, 16, 8, 8)]


@pytest.mark.parametrize("shape", SHAPES)
def test_forward_matches_oracle(shape):
    rng = np.random.default_rng(11)
    th = theta_f32(1)
    x = rng.normal(size=shape + (4,)).astype(np.float32).astype(np.float64)
    net = rf.Network()
    net.set_params(th)
    y = torch.empty(shape, dtype=torch.float32, device="cuda")
    net.forward(dev(x), y)
    yg = y.double().cpu().numpy()
    yb = NO.forward(th, x, bf16=True)[0]      # same BF16 storage points
    y64 = NO.forward(th, x)[0]                # exact FP64 network
    scale = max(np.max(np.abs(y64)), 1e-30)
    # BF16 storage rounding (unit 2^-9) that the two sides may take on
    # opposite sides of a tie, propagated through 10 layers
    assert np.max(np.abs(yg - yb)) <= 2e-2 * scale
    assert np.mean(np.abs(yg - yb)) <= 2e-3 * scale
    assert np.max(np.abs(yg - y64)) <= 5e-2 * scale


def test_params_roundtrip():
    th = W.nn_init_params(3).astype(np.float32)
    net = rf.Network()
    net.set_params(th)
    np.testing.assert_array_equal(net.get_params(), th)
    with pytest.raises(rf.RFError):
        net.set_params(np.full(rf.NN_PARAMS, np.nan, dtype=np.float32))


def _layer_slices():
    out, o = [], 0
    for ci, co in NO.LAYERS:
        out.append(slice(o, o + 27 * ci * co + co))
        o += 27 * ci * co + co
    return out


U32 = 2.0 ** -24


def _in_round_interval(got, v, e, relu=False):
    """got lies in {bf16(f(w)) : |w - v| <= e} (f = relu or identity; bf16
    rounding is monotone, so the interval's ends bound it)."""
    f = (lambda a: np.maximum(a, 0.0)) if relu else (lambda a: a)
    lo, hi = NO.bf16_round(f(v - e)), NO.bf16_round(f(v + e))
    return (got >= lo) & (got <= hi)


@pytest.mark.parametrize("shape", [(1, 5, 7, 9), (2, 4, 6, 5), (1, 3, 6, 41)])
def test_gradient_layers_match_oracle_elementwise(shape):
    """Every layer of the gradient evaluation, element by element, against
    the oracle evaluated on the GPU's own stored inputs of that layer (the
    trace of rf_nn_loss_grad): forward activations and backward output
    gradients lie within the BF16 rounding of the oracle's value widened by
    the layer's FP32 accumulation bound (2 K u sum |terms|, K terms of
    u = 2^-24), and every weight and bias gradient is within 2 M u sum |terms|
    of the oracle's FP64 contraction of the same BF16 operands over the M
    voxels."""
    rng = np.random.default_rng(12)
    th = theta_f32(2)
    x = rng.normal(size=shape + (4,)).astype(np.float32).astype(np.float64)
    tgt = rng.normal(size=shape).astype(np.float32).astype(np.float64)
    mask = (rng.random(shape) > 0.25).astype(np.float64)
    net = rf.Network()
    net.set_params(th)
    net.set_trace(True)
    L, g = net.loss_grad(dev(x), dev(tgt), dev(mask))
    g = g.astype(np.float64)
    layers = [(NO.bf16_round(Wl), bl) for Wl, bl in NO.unflatten(th)]
    absW = [np.abs(Wl) for Wl, _ in layers]
    M = int(np.prod(shape))
    tr = lambda what, i: net.trace_get(what, i, shape)
    x0 = tr("input", 0)
    assert np.all(x0[..., 4:] == 0) and np.array_equal(x0[..., :4], NO.bf16_round(x))
    x0 = x0[..., :4]
    A = [tr("block_out", i) for i in range(5)]
    U = [tr("block_mid", i) for i in range(4)]
    G = [tr("out_grad", l) for l in range(10)]
    y = tr("output", 0)[..., 0]

    def fwd(inp, li, res=None):
        Wl, bl = layers[li]
        K = 27 * Wl.shape[4] + 1 + (res is not None)
        z = NO.conv3d(inp, Wl, bl) + (0.0 if res is None else res)
        e = 2 * K * U32 * (NO.conv3d(np.abs(inp), absW[li], np.abs(bl)) + (0.0 if res is None else np.abs(res)))
        return z, e

    # forward, layer by layer from the GPU's stored inputs
    z, e = fwd(x0, 0)
    assert np.all(_in_round_interval(A[0], z, e, relu=True)), "input convolution"
    for blk in range(4):
        z, e = fwd(A[blk], 1 + 2 * blk)
        assert np.all(_in_round_interval(U[blk], z, e, relu=True)), f"block {blk + 1} conv 1"
        z, e = fwd(U[blk], 2 + 2 * blk, res=A[blk])
        assert np.all(_in_round_interval(A[blk + 1], z, e, relu=True)), f"block {blk + 1} conv 2"
    z, e = fwd(A[4], 9)
    assert np.all(np.abs(y - z[..., 0]) <= e[..., 0]), "output convolution"
    # backward: output gradients from the GPU's stored upstream values
    dy = 2.0 * (y - tgt) * mask / M
    assert np.all(G[9][..., 1:] == 0)
    assert np.all(_in_round_interval(G[9][..., 0], dy, 4 * U32 * np.abs(dy))), "loss gradient"

    def ingrad(gb, li):
        Wl = layers[li][0]
        K = 27 * Wl.shape[0]
        return NO.conv3d_input_grad(gb, Wl), 2 * K * U32 * NO.conv3d_input_grad(np.abs(gb), absW[li])

    da, e_da = ingrad(G[9][..., :1], 9)
    for blk in reversed(range(4)):
        m2 = A[blk + 1] > 0
        g2, e2 = da * m2, e_da * m2
        assert np.all(_in_round_interval(G[2 + 2 * blk], g2, e2)), f"block {blk + 1} conv 2 output gradient"
        du, e_du = ingrad(G[2 + 2 * blk], 2 + 2 * blk)
        m1 = U[blk] > 0
        assert np.all(_in_round_interval(G[1 + 2 * blk], du * m1, e_du * m1)), f"block {blk + 1} conv 1 output gradient"
        dc, e_dc = ingrad(G[1 + 2 * blk], 1 + 2 * blk)
        da = dc + g2
        e_da = e_dc + e2 + U32 * (np.abs(dc) + np.abs(g2))
    m0 = A[0] > 0
    assert np.all(_in_round_interval(G[0], da * m0, e_da * m0)), "input convolution output gradient"
    # weight and bias gradients, element by element, from the same operands
    ins = [x0] + [A[b] if l % 2 else U[b] for l, b in ((l, (l - 1) // 2) for l in range(1, 9))] + [A[4]]
    outs = G[:9] + [G[9][..., :1]]
    ref, bnd = [], []
    for l in range(10):
        dW, db = NO.conv3d_weight_grad(ins[l], outs[l])
        aW, ab = NO.conv3d_weight_grad(np.abs(ins[l]), np.abs(outs[l]))
        ref.append((dW, db))
        bnd.append((2 * M * U32 * aW + 1e-30, 2 * M * U32 * ab + 1e-30))
    ref, bnd = NO.flatten(ref), NO.flatten(bnd)
    err = np.abs(g - ref)
    assert np.all(err <= bnd), (int(np.argmax(err / bnd)), float(np.max(err / bnd)))
    # the bound is tight: a mirrored tap in one hidden layer falls far outside it
    sl = _layer_slices()[3]
    Wg = ref[sl][:27 * 32 * 32].reshape(32, 3, 3, 3, 32)
    bad = Wg[:, ::-1, ::-1, ::-1, :].ravel()
    assert np.mean(np.abs(bad - ref[sl][:27 * 32 * 32]) > bnd[sl][:27 * 32 * 32]) > 0.5
    # and the whole chain stays close to the BF16 oracle evaluated end to end
    Lb, gb = NO.loss_and_grad(th, x, tgt, mask, bf16=True)
    assert L == pytest.approx(Lb, rel=1e-2)
    assert (g @ gb) / (np.linalg.norm(g) * np.linalg.norm(gb)) >= 0.999


def test_adam_step_matches_oracle():
    rng = np.random.default_rng(13)
    shape = (1, 4, 5, 6)
    th = theta_f32(4)
    x = dev(rng.normal(size=shape + (4,)))
    tgt = dev(rng.normal(size=shape))
    net = rf.Network()
    net.set_params(th)
    _, g = net.loss_grad(x, tgt)
    lr = 1e-3
    net.train_step(x, tgt, lr=lr)
    th1 = net.get_params().astype(np.float64)
    exp, _, _ = NO.adam_step(th, g.astype(np.float64), np.zeros_like(th), np.zeros_like(th), 1, lr=lr)
    # first Adam step moves each weight by about lr sign(g); the gradient of
    # the training step differs from loss_grad's only in summation order
    big = np.abs(g) > 1e-6
    np.testing.assert_allclose(th1[big], exp[big], rtol=0, atol=1e-3 * lr + 2e-7)
    assert np.max(np.abs(th1 - th)) <= 1.01 * lr + 2e-7


def test_training_fits_a_smooth_map():
    rng = np.random.default_rng(14)
    shape = (4, 8, 8, 8)
    x = rng.normal(size=shape + (4,))
    # target: a local function of the features the network can represent
    tgt = np.tanh(x[..., 0]) * 0.5 + 0.3 * x[..., 1] - 0.2 * np.maximum(x[..., 2], 0)
    net = rf.Network()
    net.set_params(W.nn_init_params(5))
    xd, td = dev(x), dev(tgt)
    L0 = net.train_step(xd, td, lr=2e-3)
    for _ in range(150):
        L = net.train_step(xd, td, lr=2e-3, want_loss=False)
    L = net.train_step(xd, td, lr=2e-3)
    assert L < 0.1 * L0


# ---------------------------------------------------------------- solver side
def small_box(seed=3, nx=20, ny=16, nz=12):
    c = W.heterogeneous_box(nx=nx, ny=ny, nz=nz, d=0.25, seed=seed)
    return c


def masked_case():
    from tests.test_gpu_parity import masked_case as mc
    return mc()


def _oracle_features(case, h, t, dt, sc):
    nz, ny, nx = case.nz, case.ny, case.nx
    act = np.ones(case.N, bool) if case.active is None else np.asarray(case.active, bool)
    if case.Ks_cell is not None:
        Ks = np.asarray(case.Ks_cell, float)
    else:
        zone = np.zeros(case.N, int) if case.zone_of_cell is None else np.asarray(case.zone_of_cell, int)
        Ks = np.array([s["Ks"] for s in case.soils])[zone]
    lnK = np.log(np.where(act, Ks, 1.0))
    q = 0.0
    for bc in case.bcs:
        if bc.face == "zmax" and bc.type == "flux":
            i = 0
            while i + 1 < len(bc.t) and bc.t[i + 1] <= t:
                i += 1
            q = bc.v[i]
    scd = dict(h_scale=sc.h_scale, lnK_mean=sc.lnK_mean, lnK_std=sc.lnK_std, q_scale=sc.q_scale,
               t_scale=sc.t_scale, out_scale=sc.out_scale)
    return NO.features(h.reshape(nz, ny, nx), lnK.reshape(nz, ny, nx), act.reshape(nz, ny, nx), q, dt, scd), scd


@pytest.mark.parametrize("which,t", [("box", 0.0), ("box", 7 * 3600.0), ("masked", 30.0), ("masked", 60.0)])
def test_features_and_target_match_oracle(which, t):
    """Features of the current state (before and after a top-flux
    breakpoint) and of a given state; the target of a given old state."""
    case = small_box() if which == "box" else masked_case()
    sc = warmstart.scales_for(case, out_scale=2e-6, h_scale=1.5)
    s = rf.Solver.from_case(case)
    s.set_state(case.h0, t)
    dt = 17.0
    x = torch.empty((case.N, 4), dtype=torch.float32, device="cuda")
    s.ws_features(sc, t, dt, x)
    rng = np.random.default_rng(15)
    h_other = case.h0 + rng.normal(0, 0.1, case.N)
    x2 = torch.empty((case.N, 4), dtype=torch.float32, device="cuda")
    s.ws_features(sc, t, dt, x2, h=dev(h_other, torch.float64))
    tg = torch.empty(case.N, dtype=torch.float32, device="cuda")
    mk = torch.empty(case.N, dtype=torch.float32, device="cuda")
    s.ws_target(sc, dev(h_other, torch.float64), dt, tg, mk)
    torch.cuda.synchronize()
    act = np.ones(case.N, bool) if case.active is None else np.asarray(case.active, bool)
    for got, h in ((x, case.h0), (x2, h_other)):
        f_exp, scd = _oracle_features(case, np.where(act, h, 0.0), t, dt, sc)
        np.testing.assert_allclose(got.cpu().numpy().reshape(f_exp.shape), f_exp.astype(np.float32), rtol=2e-7,
                                   atol=1e-30)
    if which == "box":
        assert x.cpu().numpy().reshape(f_exp.shape)[-1, ..., 2].min() == (1.0 if t < 6 * 3600 else 0.0)
    h_new = s.get_state()[0]
    t_exp = NO.target(h_new, h_other, act, dt, scd)
    np.testing.assert_allclose(tg.cpu().numpy(), t_exp.astype(np.float32), rtol=2e-7, atol=1e-30)
    np.testing.assert_array_equal(mk.cpu().numpy(), act.astype(np.float32))


def test_warm_started_steps_match_plain_oracle():
    """Steps started from a (random, untrained) network's guess converge to
    the plain oracle's solution within the Picard tolerance's reach."""
    case = small_box(seed=5)
    fixed = dict(dt0=120.0, f_grow=1.0)
    s = rf.Solver.from_case(case, **fixed)
    o = oracle_from_case(case, **fixed)
    net = rf.Network()
    net.set_params(W.nn_init_params(6))
    sc = warmstart.scales_for(case, out_scale=1e-6)
    s.ws_attach(net, sc)
    for _ in range(6):
        si = s.step()
        oi = o.step()
        assert si.dt == pytest.approx(oi.dt, rel=1e-12)
        assert si.rejected == 0
        d = np.max(np.abs(s.get_state()[0] - o.get_state()[0]))
        assert d <= 1e-6, d
    st = s.ws_stats()
    assert st["guesses"] == 6 and st["fallbacks"] == 0
    mb = s.mass_balance()
    assert abs(mb["closure_rel"]) <= 1e-9


def test_bad_guess_falls_back_to_plain_method():
    case = small_box(seed=7)
    base = dict(dt0=60.0, f_grow=1.0)
    plain = rf.Solver.from_case(case, **base)
    p_iters = plain.step().picard
    n_max = max(p_iters, 2)
    s = rf.Solver.from_case(case, n_max=n_max, **base)
    net = rf.Network()
    th = np.zeros(rf.NN_PARAMS, dtype=np.float32)
    th[-1] = 1.0                                  # output bias: y = 1 everywhere
    net.set_params(th)
    sc = warmstart.scales_for(case, out_scale=50.0 / 60.0)   # guess = h + 50 m
    s.ws_attach(net, sc)
    info = s.step()
    st = s.ws_stats()
    assert st["guesses"] == 1 and st["fallbacks"] == 1
    assert info.rejected == 1
    f = case.params.get("f_shrink", 2.0)
    assert info.dt == pytest.approx(60.0 / f, rel=1e-12)
    o = oracle_from_case(case, dt0=60.0 / f, f_grow=1.0, n_max=n_max)
    o.step()
    assert np.max(np.abs(s.get_state()[0] - o.get_state()[0])) <= 1e-6


def test_trained_network_saves_picard_iterations():
    """Train on one seed's plain-solver snapshots with these kernels, then
    run a held-out seed with and without the warm start at a fixed step."""
    fixed = dict(dt0=300.0, f_grow=1.0)
    train_case = W.heterogeneous_box(nx=24, ny=24, nz=24, d=0.25, seed=21)
    train_case.params.update(fixed)
    sc = warmstart.scales_for(train_case)
    s = rf.Solver.from_case(train_case)
    pilot = warmstart.collect(s, train_case, sc, 8)
    sc.out_scale = warmstart.target_rms(pilot)
    s = rf.Solver.from_case(train_case)
    snaps = warmstart.collect(s, train_case, sc, 120)
    net = rf.Network()
    net.set_params(W.nn_init_params(22))
    losses = warmstart.train(net, snaps, steps=300, batch=4, lr=2e-3, log_every=100)
    assert losses[-1][1] < 0.5 * losses[0][1]

    test_case = W.heterogeneous_box(nx=24, ny=24, nz=24, d=0.25, seed=23)
    test_case.params.update(fixed)
    runs = {}
    for mode in ("plain", "warm"):
        s = rf.Solver.from_case(test_case)
        if mode == "warm":
            s.ws_attach(net, sc)
        infos = [s.step() for _ in range(60)]
        runs[mode] = (sum(i.picard for i in infos), s.get_state()[0], s.ws_stats(), [i.dt for i in infos])
    assert runs["warm"][2]["fallbacks"] == 0
    assert runs["warm"][3] == runs["plain"][3]
    assert np.max(np.abs(runs["warm"][1] - runs["plain"][1])) <= 1e-5
    # measured on GB300: 255-266 against 299 Picard iterations (11-15 % fewer)
    assert runs["warm"][0] <= 0.95 * runs["plain"][0], (runs["warm"][0], runs["plain"][0])
