"""FP64 reference of the warm-start network (TEST INFRASTRUCTURE ONLY; part of the oracle).

The network maps (asinh delta, alpha_B0, alpha_M0, a) on an n^3 periodic grid to the
screened source T = nu L(chi)/src (delta where screening is off).  Plain numpy: each 3x3x3
periodic convolution is a sum over 27 rolled copies of the input times a channel matrix,
and the backward pass is written out by the chain rule.  Layout: arrays [z, y, x, c]; conv
weights W[tap][ci][co] with tap = (dz+1)*9 + (dy+1)*3 + (dx+1) and bias b[co]; the flat
parameter vector concatenates (W, b) of the ten convolutions, then the head (w[16], b).
"""
from __future__ import annotations

import numpy as np

CONVS = [(16, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (96, 32), (32, 32), (48, 16), (16, 16)]
TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def num_params():
    return sum(27 * ci * co + co for ci, co in CONVS) + 17


def unflatten(p):
    layers, o = [], 0
    for ci, co in CONVS:
        W = p[o:o + 27 * ci * co].reshape(27, ci, co)
        o += 27 * ci * co
        b = p[o:o + co]
        o += co
        layers.append((W, b))
    head = (p[o:o + 16], p[o + 16])
    return layers, head


def conv(x, W, b):
    y = np.zeros(x.shape[:3] + (W.shape[2],))
    for t, (dz, dy, dx) in enumerate(TAPS):
        y += np.roll(x, shift=(-dz, -dy, -dx), axis=(0, 1, 2)) @ W[t]
    return y + b


def conv_bwd(x, W, dy):
    """gradients of conv(x, W, b) with respect to x, W and b given dL/dy"""
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    xf = None
    for t, (dz, dyy, dx_) in enumerate(TAPS):
        xs = np.roll(x, shift=(-dz, -dyy, -dx_), axis=(0, 1, 2))
        dW[t] = xs.reshape(-1, x.shape[3]).T @ dy.reshape(-1, dy.shape[3])
        dx += np.roll(dy @ W[t].T, shift=(dz, dyy, dx_), axis=(0, 1, 2))
    return dx, dW, dy.sum(axis=(0, 1, 2))


def pool(x):
    n = x.shape[0]
    return x.reshape(n // 2, 2, n // 2, 2, n // 2, 2, -1).mean(axis=(1, 3, 5))


def pool_bwd(d):
    return np.repeat(np.repeat(np.repeat(d, 2, 0), 2, 1), 2, 2) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def up_bwd(d):
    n = d.shape[0]
    return d.reshape(n // 2, 2, n // 2, 2, n // 2, 2, -1).sum(axis=(1, 3, 5))


def relu(z):
    return np.maximum(z, 0.0)


def pack_input(delta, aB0, aM0, a):
    n = delta.shape[0]
    x = np.zeros((n, n, n, 16))
    x[..., 0] = np.arcsinh(delta)
    x[..., 1], x[..., 2], x[..., 3] = aB0, aM0, a
    return x


def forward(p, delta, aB0, aM0, a):
    L, (hw, hb) = unflatten(np.asarray(p, dtype=np.float64))
    s = {}
    s["in"] = pack_input(delta, aB0, aM0, a)
    s["y0"] = relu(conv(s["in"], *L[0]))
    s["y1"] = relu(conv(s["y0"], *L[1]))
    s["p1"] = pool(s["y1"])
    s["y2"] = relu(conv(s["p1"], *L[2]))
    s["y3"] = relu(conv(s["y2"], *L[3]))
    s["p2"] = pool(s["y3"])
    s["y4"] = relu(conv(s["p2"], *L[4]))
    s["y5"] = relu(conv(s["y4"], *L[5]))
    s["cat2"] = np.concatenate([up(s["y5"]), s["y3"]], axis=3)
    s["y6"] = relu(conv(s["cat2"], *L[6]))
    s["y7"] = relu(conv(s["y6"], *L[7]))
    s["cat1"] = np.concatenate([up(s["y7"]), s["y1"]], axis=3)
    s["y8"] = relu(conv(s["cat1"], *L[8]))
    s["y9"] = relu(conv(s["y8"], *L[9]))
    s["out"] = s["y9"] @ hw + hb
    return s["out"], s


def loss_grad(p, delta, target, aB0, aM0, a):
    """loss = mean((T_hat - target)^2) and its gradient with respect to the flat parameters"""
    p = np.asarray(p, dtype=np.float64)
    L, (hw, hb) = unflatten(p)
    out, s = forward(p, delta, aB0, aM0, a)
    V = out.size
    diff = out - target
    loss = float((diff * diff).mean())
    g = 2.0 * diff / V
    grads = [None] * 10
    ghw = np.einsum("zyx,zyxc->c", g, s["y9"])
    ghb = g.sum()
    d = g[..., None] * hw * (s["y9"] > 0)                       # d pre-activation of c9
    dx, dW, db = conv_bwd(s["y8"], L[9][0], d); grads[9] = (dW, db)
    d = dx * (s["y8"] > 0)                                      # c8
    dx, dW, db = conv_bwd(s["cat1"], L[8][0], d); grads[8] = (dW, db)
    dcat1 = dx
    d = up_bwd(dcat1[..., :32]) * (s["y7"] > 0)                 # c7
    dx, dW, db = conv_bwd(s["y6"], L[7][0], d); grads[7] = (dW, db)
    d = dx * (s["y6"] > 0)                                      # c6
    dx, dW, db = conv_bwd(s["cat2"], L[6][0], d); grads[6] = (dW, db)
    dcat2 = dx
    d = up_bwd(dcat2[..., :64]) * (s["y5"] > 0)                 # c5
    dx, dW, db = conv_bwd(s["y4"], L[5][0], d); grads[5] = (dW, db)
    d = dx * (s["y4"] > 0)                                      # c4
    dx, dW, db = conv_bwd(s["p2"], L[4][0], d); grads[4] = (dW, db)
    dy3 = dcat2[..., 64:] + pool_bwd(dx)
    d = dy3 * (s["y3"] > 0)                                     # c3
    dx, dW, db = conv_bwd(s["y2"], L[3][0], d); grads[3] = (dW, db)
    d = dx * (s["y2"] > 0)                                      # c2
    dx, dW, db = conv_bwd(s["p1"], L[2][0], d); grads[2] = (dW, db)
    dy1 = dcat1[..., 32:] + pool_bwd(dx)
    d = dy1 * (s["y1"] > 0)                                     # c1
    dx, dW, db = conv_bwd(s["y0"], L[1][0], d); grads[1] = (dW, db)
    d = dx * (s["y0"] > 0)                                      # c0
    dx, dW, db = conv_bwd(s["in"], L[0][0], d); grads[0] = (dW, db)
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads] + [ghw, [ghb]])
    return loss, flat


def init_params(seed):
    """He-normal weights for the ReLU layers, zero biases, small head (seeded numpy)."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, (ci, co) in enumerate(CONVS):
        fan_in = 27 * (4 if i == 0 else ci)
        parts.append(rng.standard_normal(27 * ci * co) * np.sqrt(2.0 / fan_in))
        parts.append(np.zeros(co))
    parts.append(rng.standard_normal(16) * np.sqrt(1.0 / 16))
    parts.append([0.0])
    return np.concatenate(parts)
