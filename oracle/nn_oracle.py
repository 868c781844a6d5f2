"""Plain FP64 CPU oracle of the learned warm start (network, loss, Adam,
features, guess).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` (and nothing else).  It
shares no code with the CUDA path.

The paper (Orgogozo et al., arXiv:1809.10895) has no learned component: it
starts every Picard iteration sequence of Sec. 2.2 from the previous time
level.  This module writes out, in numpy, what the warm start computes:

* a 3-D convolutional residual network: an input convolution 4 -> 32, four
  residual blocks of two 3x3x3 convolutions 32 -> 32 with ReLU (the block's
  input is added before the second ReLU, He et al. 2016), an output
  convolution 32 -> 1.  All convolutions are 3x3x3, stride 1, zero padding 1,
  cross-correlation ``out[v] = b + sum_tap W[:, tap] in[v + tap]``;
* the masked mean-squared error, its gradient by reverse-mode
  differentiation written out layer by layer, and Adam (Kingma & Ba 2015);
* the solver-facing features and the guess ``h^n + y * out_scale * dt``.

Arrays are channels-last: ``x[b, z, y, x, c]``.  A weight is
``W[cout, dz, dy, dx, cin]`` (``dz = 0`` is the -1 offset).  The flat
parameter vector lists, layer by layer, ``W.ravel()`` then ``b``.

``bf16=True`` rounds at the points where the BF16 network stores values:
inputs, weights and hidden activations, and the output gradients of each
convolution, which enter both its input-gradient and its weight-gradient
contraction.  Everything else stays FP64.
"""
from __future__ import annotations

import numpy as np

C_IN, C_HID, C_OUT = 4, 32, 1
N_BLOCKS = 4
# (cin, cout) per convolution: input conv, 2 per residual block, output conv
LAYERS = [(C_IN, C_HID)] + [(C_HID, C_HID)] * (2 * N_BLOCKS) + [(C_HID, C_OUT)]


def n_params() -> int:
    return sum(27 * ci * co + co for ci, co in LAYERS)


def unflatten(theta: np.ndarray):
    """Flat vector -> list of (W, b)."""
    out, o = [], 0
    for ci, co in LAYERS:
        nW = 27 * ci * co
        W = theta[o:o + nW].reshape(co, 3, 3, 3, ci)
        o += nW
        b = theta[o:o + co]
        o += co
        out.append((W, b))
    assert o == theta.shape[0]
    return out


def flatten(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), through float32."""
    f = np.asarray(a, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


# ------------------------------------------------------------------ layers
def shifted(x: np.ndarray, dz: int, dy: int, dx: int) -> np.ndarray:
    """s[b, z, y, x] = x[b, z + dz, y + dy, x + dx], zero outside."""
    B, D, H, W, C = x.shape
    s = np.zeros_like(x)
    zs, zd = (slice(dz, D), slice(0, D - dz)) if dz >= 0 else (slice(0, D + dz), slice(-dz, D))
    ys, yd = (slice(dy, H), slice(0, H - dy)) if dy >= 0 else (slice(0, H + dy), slice(-dy, H))
    xs, xd = (slice(dx, W), slice(0, W - dx)) if dx >= 0 else (slice(0, W + dx), slice(-dx, W))
    s[:, zd, yd, xd, :] = x[:, zs, ys, xs, :]
    return s


TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def conv3d(x: np.ndarray, W: np.ndarray, b) -> np.ndarray:
    """out[v, co] = b[co] + sum_tap sum_ci W[co, tap, ci] x[v + tap, ci]."""
    out = np.zeros(x.shape[:4] + (W.shape[0],))
    for dz, dy, dx in TAPS:
        out += shifted(x, dz, dy, dx) @ W[:, dz + 1, dy + 1, dx + 1, :].T
    if b is not None:
        out += b
    return out


def conv3d_input_grad(g: np.ndarray, W: np.ndarray) -> np.ndarray:
    """d(sum g . conv3d(x))/dx: each tap sends g back by the opposite offset."""
    out = np.zeros(g.shape[:4] + (W.shape[4],))
    for dz, dy, dx in TAPS:
        out += shifted(g, -dz, -dy, -dx) @ W[:, dz + 1, dy + 1, dx + 1, :]
    return out


def conv3d_weight_grad(x: np.ndarray, g: np.ndarray):
    """dW[co, tap, ci] = sum_v g[v, co] x[v + tap, ci]; db = sum_v g[v]."""
    co, ci = g.shape[-1], x.shape[-1]
    dW = np.zeros((co, 3, 3, 3, ci))
    g2 = g.reshape(-1, co)
    for dz, dy, dx in TAPS:
        dW[:, dz + 1, dy + 1, dx + 1, :] = g2.T @ shifted(x, dz, dy, dx).reshape(-1, ci)
    return dW, g2.sum(axis=0)


# ------------------------------------------------------------------ network
def forward(theta: np.ndarray, x: np.ndarray, bf16: bool = False):
    """Network output y[b, z, y, x] and the stored activations."""
    rnd = bf16_round if bf16 else (lambda a: a)
    layers = [(rnd(W), b) for W, b in unflatten(np.asarray(theta, dtype=np.float64))]
    x0 = rnd(x)
    a = rnd(np.maximum(conv3d(x0, *layers[0]), 0.0))
    acts = {"x0": x0, "a": [a], "u": []}
    for blk in range(N_BLOCKS):
        W1, b1 = layers[1 + 2 * blk]
        W2, b2 = layers[2 + 2 * blk]
        u = rnd(np.maximum(conv3d(a, W1, b1), 0.0))
        a = rnd(np.maximum(conv3d(u, W2, b2) + a, 0.0))
        acts["u"].append(u)
        acts["a"].append(a)
    y = conv3d(a, *layers[-1])[..., 0]
    return y, acts, layers


def loss(y: np.ndarray, target: np.ndarray, mask=None) -> float:
    """L = (1/M) sum_v mask_v (y_v - t_v)^2 over all M voxels."""
    d = y - target
    if mask is not None:
        d = d * mask
    return float(np.sum(d * d) / d.size)


def loss_and_grad(theta: np.ndarray, x: np.ndarray, target: np.ndarray, mask=None, bf16: bool = False):
    """L and dL/dtheta (flat, the parameter order of ``flatten``)."""
    rnd = bf16_round if bf16 else (lambda a: a)
    y, acts, layers = forward(theta, x, bf16)
    d = y - target
    if mask is not None:
        d = d * mask
    L = float(np.sum(d * d) / d.size)
    dy = 2.0 * d / d.size
    if mask is not None:
        dy = dy * mask
    dy = dy[..., None]
    grads = [None] * len(layers)
    a = acts["a"][-1]
    grads[-1] = conv3d_weight_grad(a, rnd(dy))
    da = conv3d_input_grad(rnd(dy), layers[-1][0])
    for blk in reversed(range(N_BLOCKS)):
        a_out, a_in, u = acts["a"][blk + 1], acts["a"][blk], acts["u"][blk]
        W1 = layers[1 + 2 * blk][0]
        W2 = layers[2 + 2 * blk][0]
        g2 = da * (a_out > 0)                       # through the second ReLU
        grads[2 + 2 * blk] = conv3d_weight_grad(u, rnd(g2))
        du = conv3d_input_grad(rnd(g2), W2)
        g1 = du * (u > 0)
        grads[1 + 2 * blk] = conv3d_weight_grad(a_in, rnd(g1))
        da = conv3d_input_grad(rnd(g1), W1) + g2    # conv branch + identity branch
    g0 = da * (acts["a"][0] > 0)
    grads[0] = conv3d_weight_grad(acts["x0"], rnd(g0))
    return L, flatten(grads)


def adam_step(theta, grad, m, v, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1); t counts from 1."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


# ------------------------------------------------------------------ solver side
def features(h, lnKs, active, q_top, dt, scales) -> np.ndarray:
    """Network inputs of one mesh state, shape (nz, ny, nx, 4).

    h, lnKs, active: (nz, ny, nx) arrays (z up).  Channels: h / h_scale;
    (ln Ks - lnK_mean) / lnK_std; q_top / q_scale on cells whose +z neighbour
    is outside the mesh or inactive, else 0; ln(dt / t_scale).  Inactive
    cells are all zero.
    """
    h = np.asarray(h, dtype=np.float64)
    act = np.asarray(active, dtype=bool)
    top = np.ones_like(act)
    top[:-1] = ~act[1:]
    f = np.zeros(h.shape + (4,))
    f[..., 0] = h / scales["h_scale"]
    f[..., 1] = (lnKs - scales["lnK_mean"]) / scales["lnK_std"]
    f[..., 2] = np.where(top, q_top / scales["q_scale"], 0.0)
    f[..., 3] = np.log(dt / scales["t_scale"])
    f[~act] = 0.0
    return f


def guess(h, y, active, dt, scales) -> np.ndarray:
    """Initial Picard iterate: h + y out_scale dt on active cells."""
    g = np.array(h, dtype=np.float64)
    act = np.asarray(active, dtype=bool)
    g[act] += y[act] * scales["out_scale"] * dt
    return g


def target(h_new, h_old, active, dt, scales) -> np.ndarray:
    """Training target: (h^{n+1} - h^n) / (out_scale dt), 0 on inactive cells."""
    t = (np.asarray(h_new) - np.asarray(h_old)) / (scales["out_scale"] * dt)
    return np.where(np.asarray(active, dtype=bool), t, 0.0)
