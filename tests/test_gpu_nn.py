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


@pytest.mark.parametrize("shape", [(1, 5, 7, 9), (2, 4, 6, 5)])
def test_gradient_matches_oracle(shape):
    rng = np.random.default_rng(12)
    th = theta_f32(2)
    x = rng.normal(size=shape + (4,)).astype(np.float32).astype(np.float64)
    tgt = rng.normal(size=shape).astype(np.float32).astype(np.float64)
    mask = (rng.random(shape) > 0.25).astype(np.float64)
    net = rf.Network()
    net.set_params(th)
    L, g = net.loss_grad(dev(x), dev(tgt), dev(mask))
    Lb, gb = NO.loss_and_grad(th, x, tgt, mask, bf16=True)
    L64, g64 = NO.loss_and_grad(th, x, tgt, mask)
    assert L == pytest.approx(Lb, rel=1e-2)
    g = g.astype(np.float64)
    for sl in _layer_slices():
        ref = gb[sl]
        rel = np.linalg.norm(g[sl] - ref) / max(np.linalg.norm(ref), 1e-30)
        assert rel <= 3e-2, (sl, rel)
        rel64 = np.linalg.norm(g[sl] - g64[sl]) / max(np.linalg.norm(g64[sl]), 1e-30)
        assert rel64 <= 1e-1, (sl, rel64)
    cos = g @ gb / (np.linalg.norm(g) * np.linalg.norm(gb))
    assert cos >= 0.999


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
