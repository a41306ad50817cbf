"""FP64 CPU oracle of the fluence surrogate: a 3D U-Net on voxel masks.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
CPU-baseline leg of the benchmark may import this module.  It shares no code
with the CUDA library; the two meet only through seeded inputs.

The surrogate maps a pore mask plus the solid optics (mu_s h, mu_a h, g) to
the log of the voxel fluence that the Monte Carlo engine tallies (Sec. 2.5-2.6
estimators), so that design sweeps over masks (Sec. 5) can be screened
without a full photon run.  The paper defines no network; this module is the
plain definition the GPU kernels must reproduce, written with numpy matmuls
as the only library step.

Tensors are channels-last float64 arrays (B, D, H, W, C).

  conv3  3x3x3, stride 1, zero padding 1:
           y[v] = b + sum_t x[v + t] @ W[t],  t = (dz, dy, dx) in {-1, 0, 1}^3,
           tap index (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);  W: (27, Cin, Cout)
  down   2x2x2, stride 2 (D, H, W even):
           y[v] = b + sum_o x[2v + o] @ W[o],  o = (oz, oy, ox) in {0, 1}^3,
           tap index oz * 4 + oy * 2 + ox;  W: (8, Cin, Cout)
  up     transposed 2x2x2, stride 2:  y[2v + o] = b + x[v] @ W[o];  W: (8, Cin, Cout)
  head   p[v] = c + x[v] . h  (one output channel, float)
  loss   mean over every voxel of every sample of w (p - target)^2, with
         w = 1 (plain), or, fluence-weighted, w = exp(target) divided by the
         mean of exp(target) over the voxels of the same sample: the target
         is a log fluence, so this weighs each voxel's log error by its
         fluence, as Eq. RMSw weighs depth layers (weights average to 1)

Network with base width c0 (widths c0, 2c0, 4c0, 8c0 on four levels):

  e0a = relu(conv3(x))          e0b = relu(conv3(e0a))              level 0
  d1  = relu(down(e0b))         e1a, e1b = two relu(conv3) at 2c0   level 1
  d2  = relu(down(e1b))         e2a, e2b at 4c0                     level 2
  d3  = relu(down(e2b))         b1, b2 at 8c0                       level 3
  u2  = up(b2)                  c2a = relu(conv3([u2, e2b])), c2b
  u1  = up(c2b)                 c1a = relu(conv3([u1, e1b])), c1b
  u0  = up(c1b)                 c0a = relu(conv3([u0, e0b])), c0b
  p   = head(c0b)

([a, b] is the channel concatenation, a first.)  Backward passes are the chain
rule written out layer by layer; the tests pin them against central finite
differences and the adjoint identities, not against themselves.
"""
from __future__ import annotations

import math

import numpy as np

N_FEATURES = 16          # input channels (see pack_input)


# ------------------------------------------------------------------ layers --

def _taps3():
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _taps2():
    return [(oz, oy, ox) for oz in (0, 1) for oy in (0, 1) for ox in (0, 1)]


def _mm(x, w):
    """x (..., Cin) @ w (Cin, Cout) in float64."""
    return np.tensordot(x, w, axes=([x.ndim - 1], [0]))


def conv3(x, w, b=None):
    B, D, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((B, D, H, W, w.shape[2]))
    for t, (dz, dy, dx) in enumerate(_taps3()):
        y += _mm(xp[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W, :], w[t])
    return y if b is None else y + b


def conv3_dgrad(dy, w):
    """Adjoint of conv3 in x: dx[v] = sum_t dy[v - t] @ W[t]^T."""
    B, D, H, W, _ = dy.shape
    dyp = np.pad(dy, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    dx = np.zeros((B, D, H, W, w.shape[1]))
    for t, (dz, dy_, dx_) in enumerate(_taps3()):
        dx += _mm(dyp[:, 1 - dz:1 - dz + D, 1 - dy_:1 - dy_ + H, 1 - dx_:1 - dx_ + W, :], w[t].T)
    return dx


def conv3_wgrad(x, dy):
    """dW[t] = sum_v x[v + t]^T dy[v] (x zero outside), db = sum_v dy[v]."""
    B, D, H, W, C = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    g = dy.reshape(-1, dy.shape[-1])
    dw = np.zeros((27, C, dy.shape[-1]))
    for t, (dz, dy_, dx_) in enumerate(_taps3()):
        xs = xp[:, 1 + dz:1 + dz + D, 1 + dy_:1 + dy_ + H, 1 + dx_:1 + dx_ + W, :]
        dw[t] = xs.reshape(-1, C).T @ g
    return dw, g.sum(axis=0)


def down(x, w, b=None):
    y = 0.0
    for o, (oz, oy, ox) in enumerate(_taps2()):
        y = y + _mm(x[:, oz::2, oy::2, ox::2, :], w[o])
    return y if b is None else y + b


def down_dgrad(dy, w):
    B, D, H, W, _ = dy.shape
    dx = np.zeros((B, 2 * D, 2 * H, 2 * W, w.shape[1]))
    for o, (oz, oy, ox) in enumerate(_taps2()):
        dx[:, oz::2, oy::2, ox::2, :] = _mm(dy, w[o].T)
    return dx


def down_wgrad(x, dy):
    g = dy.reshape(-1, dy.shape[-1])
    dw = np.zeros((8, x.shape[-1], dy.shape[-1]))
    for o, (oz, oy, ox) in enumerate(_taps2()):
        dw[o] = x[:, oz::2, oy::2, ox::2, :].reshape(-1, x.shape[-1]).T @ g
    return dw, g.sum(axis=0)


def up(x, w, b=None):
    B, D, H, W, _ = x.shape
    y = np.zeros((B, 2 * D, 2 * H, 2 * W, w.shape[2]))
    for o, (oz, oy, ox) in enumerate(_taps2()):
        y[:, oz::2, oy::2, ox::2, :] = _mm(x, w[o])
    return y if b is None else y + b


def up_dgrad(dy, w):
    dx = 0.0
    for o, (oz, oy, ox) in enumerate(_taps2()):
        dx = dx + _mm(dy[:, oz::2, oy::2, ox::2, :], w[o].T)
    return dx


def up_wgrad(x, dy):
    xf = x.reshape(-1, x.shape[-1])
    dw = np.zeros((8, x.shape[-1], dy.shape[-1]))
    for o, (oz, oy, ox) in enumerate(_taps2()):
        dw[o] = xf.T @ dy[:, oz::2, oy::2, ox::2, :].reshape(-1, dy.shape[-1])
    return dw, dy.reshape(-1, dy.shape[-1]).sum(axis=0)


def relu(x):
    return np.maximum(x, 0.0)


# ----------------------------------------------------------------- network --

def layer_table(c0: int, cin: int = N_FEATURES):
    """(name, kind, input channels, output channels, relu) in forward order.
    A conv3 whose name ends in 'a' on the decoder side reads [up, skip]."""
    c1, c2, c3 = 2 * c0, 4 * c0, 8 * c0
    return [
        ("e0a", "conv3", cin, c0, True), ("e0b", "conv3", c0, c0, True),
        ("d1", "down", c0, c1, True), ("e1a", "conv3", c1, c1, True), ("e1b", "conv3", c1, c1, True),
        ("d2", "down", c1, c2, True), ("e2a", "conv3", c2, c2, True), ("e2b", "conv3", c2, c2, True),
        ("d3", "down", c2, c3, True), ("b1", "conv3", c3, c3, True), ("b2", "conv3", c3, c3, True),
        ("u2", "up", c3, c2, False), ("c2a", "conv3", 2 * c2, c2, True), ("c2b", "conv3", c2, c2, True),
        ("u1", "up", c2, c1, False), ("c1a", "conv3", 2 * c1, c1, True), ("c1b", "conv3", c1, c1, True),
        ("u0", "up", c1, c0, False), ("c0a", "conv3", 2 * c0, c0, True), ("c0b", "conv3", c0, c0, True),
    ]


SKIP_OF = {"c2a": ("u2", "e2b"), "c1a": ("u1", "e1b"), "c0a": ("u0", "e0b")}
N_TAPS = {"conv3": 27, "down": 8, "up": 8}


def init_params(c0: int, seed: int, cin: int = N_FEATURES):
    """He-normal weights (fan-in = taps x input channels), small biases."""
    rng = np.random.default_rng(seed)
    params = {}
    for name, kind, ci, co, _ in layer_table(c0, cin):
        taps = N_TAPS[kind]
        fan_in = (taps if kind != "up" else 1) * ci
        params[name] = (rng.standard_normal((taps, ci, co)) * math.sqrt(2.0 / fan_in),
                        rng.uniform(-0.05, 0.05, co))
    params["head"] = (rng.standard_normal(c0) * math.sqrt(1.0 / c0), np.array(rng.uniform(-0.05, 0.05)))
    return params


def forward(params, x, c0: int):
    """Returns (prediction (B, D, H, W), cache of every layer output)."""
    act = {"x": x}
    prev = "x"
    for name, kind, _, _, use_relu in layer_table(c0, x.shape[-1]):
        w, b = params[name]
        if name in SKIP_OF:
            u, s = SKIP_OF[name]
            inp = np.concatenate([act[u], act[s]], axis=-1)
        else:
            inp = act[prev]
        y = {"conv3": conv3, "down": down, "up": up}[kind](inp, w, b)
        act[name] = relu(y) if use_relu else y
        prev = name
    h, c = params["head"]
    return _mm(act[prev], h[:, None])[..., 0] + c, act


def loss_weights(target, fluence_weighted: bool = False):
    """Per-voxel loss weights: ones, or exp(target) over its sample's mean."""
    if not fluence_weighted:
        return np.ones_like(target)
    e = np.exp(target)
    mean = e.reshape(e.shape[0], -1).mean(axis=1)
    return e / mean.reshape((-1,) + (1,) * (target.ndim - 1))


def loss(pred, target, fluence_weighted: bool = False):
    return float(np.mean(loss_weights(target, fluence_weighted) * (pred - target) ** 2))


def backward(params, act, pred, target, c0: int, fluence_weighted: bool = False):
    """Gradients of loss(pred, target) for every parameter, by the chain rule."""
    table = layer_table(c0, act["x"].shape[-1])
    n = pred.size
    dp = 2.0 * loss_weights(target, fluence_weighted) * (pred - target) / n
    h, _ = params["head"]
    last = table[-1][0]
    grads = {"head": ((act[last] * dp[..., None]).reshape(-1, act[last].shape[-1]).sum(0),
                      np.array(dp.sum()))}
    # gradient w.r.t. each layer's output (post-activation)
    dout = {last: dp[..., None] * h}
    inputs = {}
    prev = "x"
    for name, _, _, _, _ in table:
        inputs[name] = SKIP_OF.get(name, (prev,))
        prev = name
    for name, kind, ci, co, use_relu in reversed(table):
        g = dout.pop(name)
        if use_relu:
            g = g * (act[name] > 0)
        w, _ = params[name]
        srcs = inputs[name]
        xin = np.concatenate([act[s] for s in srcs], axis=-1) if len(srcs) > 1 else act[srcs[0]]
        if kind == "conv3":
            dw, db = conv3_wgrad(xin, g)
            dx = conv3_dgrad(g, w)
        elif kind == "down":
            dw, db = down_wgrad(xin, g)
            dx = down_dgrad(g, w)
        else:
            dw, db = up_wgrad(xin, g)
            dx = up_dgrad(g, w)
        grads[name] = (dw, db)
        off = 0
        for s in srcs:
            cs = act[s].shape[-1]
            part = dx[..., off:off + cs]
            off += cs
            if s == "x":
                continue
            dout[s] = dout[s] + part if s in dout else part
    return grads


# ---------------------------------------------------------------- optimiser --

def adam_step(p, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma and Ba 2015, Algorithm 1); returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------------- inputs and targets --

def pack_input(mask, mus, mua, g):
    """Features per voxel, channels-last (B, D, H, W, 16):
    0 pore indicator, 1 solid indicator, 2 ln(mu_s h), 3 ln(mu_a h) / 4, 4 g,
    5 depth (z + 1/2) / D, 6 -mu_eff (z + 1/2) / 8, 7 porosity phi, 8..15 zero.
    phi is the pore fraction of the sample's mask; mu_eff = sqrt(3 mu_a' (mu_a'
    + mu_s' (1 - g))) is the diffusion-theory attenuation (Sec. 2.4: kappa =
    sqrt(mu_a / D), D = 1 / (3 (mu_a + mu_s'))) of the medium scaled to its
    solid fraction, mu' = (1 - phi) mu (Eq. EMA_scaling).  mask: (B, D, H, W),
    1 = pore."""
    m = np.asarray(mask, dtype=np.float64)
    B, D, H, W = m.shape
    x = np.zeros((B, D, H, W, N_FEATURES))
    x[..., 0] = m
    x[..., 1] = 1.0 - m
    zc = np.arange(D) + 0.5
    for b in range(B):
        phi = m[b].mean()
        ma = (1.0 - phi) * mua[b]
        msp = (1.0 - phi) * mus[b] * (1.0 - g[b])
        mu_eff = math.sqrt(3.0 * ma * (ma + msp))
        x[b, ..., 2] = math.log(mus[b])
        x[b, ..., 3] = math.log(mua[b]) / 4.0
        x[b, ..., 4] = g[b]
        x[b, ..., 6] = (-mu_eff * zc / 8.0)[:, None, None]
        x[b, ..., 7] = phi
    x[..., 5] = (zc / D)[None, :, None, None]
    return x


def log_fluence(raw_field, nx: int, ny: int, n_photons: int, floor: float = 1e-6):
    """ln max(Phi/S0, floor) from a Q32.32 track-length field:
    Phi/S0 = F nx ny / N per voxel (steady-state normalisation, Sec. 2.6)."""
    phi = np.asarray(raw_field, dtype=np.float64) / 2.0 ** 32 * nx * ny / n_photons
    return np.log(np.maximum(phi, floor))


def phase_profiles(log_phi, mask):
    """Per-phase depth profiles of exp(log_phi): (B, 2, D) mean over each z
    layer of the solid (row 0) and pore (row 1) voxels; NaN where empty."""
    phi = np.exp(np.asarray(log_phi, dtype=np.float64))
    m = np.asarray(mask).astype(bool)
    out = np.full((phi.shape[0], 2, phi.shape[1]), np.nan)
    for ph, sel in ((0, ~m), (1, m)):
        cnt = sel.sum(axis=(2, 3))
        s = (phi * sel).sum(axis=(2, 3))
        with np.errstate(invalid="ignore", divide="ignore"):
            out[:, ph, :] = np.where(cnt > 0, s / np.maximum(cnt, 1), np.nan)
    return out
