"""Learned warm start: data generation, training and checkpoints of the warm-start network.

Orchestration only; every step runs in the CUDA library.  Training pairs come from the
library's own solver: seeded fields on the GPU (lognormal with P ~ k^-2 and Zel'dovich
particles with P ~ k^-1.5, deposited by pm_deposit_cic), parameters drawn like the batched
configuration (alpha_B0 ~ U[-2,0], alpha_M0 ~ U[0,1], a ~ U[0.3,1], near-singular draws
redrawn), chi solved to relative residual 1e-8, and the target T = nu L(chi)/src.

Checkpoint format: a little-endian float32 vector of the flat parameters in a file
`<name>.bin` plus `<name>.json` with {"format": "pmeft-unet", "version": 1, "count": N,
"trained_on": ..., "loss_history": [...]}.

    python -m paper_2604_15434_gb300.learned train --pairs 2000 --n 128 --epochs 4 --out weights/unet_128
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import api

WEIGHTS_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights")
CONV_SHAPES = [(16, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (96, 32), (32, 32), (48, 16), (16, 16)]


def init_params(seed: int) -> np.ndarray:
    """He-normal convolution weights (fan-in of the real input channels), zero biases,
    and a head that starts as T_hat = channel average of the last layer (seeded numpy)."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, (ci, co) in enumerate(CONV_SHAPES):
        fan_in = 27 * (4 if i == 0 else ci)
        parts.append(rng.standard_normal(27 * ci * co) * math.sqrt(2.0 / fan_in))
        parts.append(np.zeros(co))
    parts.append(rng.standard_normal(16) * math.sqrt(1.0 / 16))
    parts.append([0.0])
    return np.concatenate(parts).astype(np.float32)


def save(net: api.UNet, path: str, meta: dict | None = None):
    p = net.get_params()
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    p.astype("<f4").tofile(path + ".bin")
    info = {"format": "pmeft-unet", "version": 1, "count": int(p.size)}
    info.update(meta or {})
    with open(path + ".json", "w") as f:
        json.dump(info, f, indent=1)


def load_params(path: str) -> np.ndarray:
    with open(path + ".json") as f:
        info = json.load(f)
    if info.get("format") != "pmeft-unet":
        raise ValueError(f"{path}.json is not a pmeft-unet checkpoint")
    p = np.fromfile(path + ".bin", dtype="<f4")
    if p.size != info["count"]:
        raise ValueError("checkpoint size mismatch")
    return p


def _gpu_gaussian(n, slope, sigma, gen, dev):
    w = torch.randn((n, n, n), generator=gen, device=dev, dtype=torch.float64)
    m = torch.fft.fftfreq(n, device=dev, dtype=torch.float64) * n
    mr = torch.fft.rfftfreq(n, device=dev, dtype=torch.float64) * n
    k2 = m[:, None, None] ** 2 + m[None, :, None] ** 2 + mr[None, None, :] ** 2
    amp = torch.where(k2 > 0, k2.clamp(min=1e-30) ** (slope / 4.0), torch.zeros_like(k2))
    g = torch.fft.irfftn(torch.fft.rfftn(w) * amp, s=(n, n, n))
    g = g - g.mean()
    return g * (sigma / g.std()), k2


def gpu_field(n, kind, sigma, gen, dev, ctx):
    """A seeded density contrast on the GPU: 'lognormal' (P ~ k^-2) or 'zeldovich' (P ~ k^-1.5)."""
    if kind == "lognormal":
        g, _ = _gpu_gaussian(n, -2.0, sigma, gen, dev)
        rho = torch.exp(g)
        return rho / rho.mean() - 1.0
    d, k2 = _gpu_gaussian(n, -1.5, sigma, gen, dev)
    dk = torch.fft.rfftn(d)
    m = torch.fft.fftfreq(n, device=dev, dtype=torch.float64) * n
    mr = torch.fft.rfftfreq(n, device=dev, dtype=torch.float64) * n
    kk = (2 * math.pi) ** 2 * k2
    kk[0, 0, 0] = 1.0
    q = (torch.arange(n, device=dev, dtype=torch.float64) + 0.5) / n
    pos = torch.empty((3, n ** 3), device=dev, dtype=torch.float64)
    for row, kv in ((0, mr[None, None, :]), (1, m[None, :, None]), (2, m[:, None, None])):
        disp = torch.fft.irfftn(1j * (2 * math.pi * kv) * dk / kk, s=(n, n, n))
        base = [q[None, None, :], q[None, :, None], q[:, None, None]][row].expand(n, n, n)
        x = (base + disp).reshape(-1)
        x = x - torch.floor(x)
        x[x >= 1.0] = 0.0
        pos[row] = x
    return api.pm_deposit_cic(pos, n, ctx=ctx)


def sample_params(rng):
    while True:
        aB, aM, a = rng.uniform(-2.0, 0.0), rng.uniform(0.0, 1.0), rng.uniform(0.3, 1.0)
        c = api.coefficients(aB, aM, a)
        if abs(c["nu"]) >= 0.1 and abs(c["mu_chi"]) <= 4.0 and c["xi"] != 0.0:
            return aB, aM, a


def make_pairs(count, n, seed, ctx, log=print):
    """count training pairs (delta, params, T) generated and solved on the GPU; deltas kept
    in FP64, targets in FP32, all resident on the device."""
    dev = ctx.device
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    rng = np.random.default_rng(seed)
    solver = api.Context(dev.index, ctx.stream, precision=1, max_cycles=100)
    pairs = []
    t0 = time.time()
    for i in range(count):
        kind = "lognormal" if i % 2 == 0 else "zeldovich"
        sigma = rng.uniform(1.0, 1.8) if kind == "lognormal" else rng.uniform(0.5, 2.0)
        delta = gpu_field(n, kind, sigma, gen, dev, solver)
        aB, aM, a = sample_params(rng)
        try:
            chi, info = api.scalar_mg_solve(delta, aB, aM, a, 1e-8, ctx=solver)
        except api.PMError:
            continue
        T = api.unet_target(chi, aB, aM, a, ctx=solver)
        pairs.append((delta, (aB, aM, a), T))
        if log and (i + 1) % 200 == 0:
            log(f"pairs {i + 1}/{count} ({time.time() - t0:.0f} s)")
    return pairs


def train(net, pairs, epochs, lr=1e-3, batch=8, seed=0, log=print, decay=0.5):
    """Adam over the pairs in shuffled mini-batches; the step size is lr * decay^epoch."""
    rng = np.random.default_rng(seed)
    hist = []
    step = 0
    for ep in range(epochs):
        order = rng.permutation(len(pairs))
        tot = 0.0
        for j, i in enumerate(order):
            delta, (aB, aM, a), T = pairs[i]
            tot += net.loss_grad(delta, T, aB, aM, a) / batch
            if (j + 1) % batch == 0:
                step += 1
                net.adam_step(lr * (decay ** ep))
        hist.append(tot / max(1, len(order) // batch))
        if log:
            log(f"epoch {ep}: mean loss {hist[-1]:.5f}")
    return hist


def linear_loss(pairs):
    """The loss of T_hat = delta (the linear solution's screened source), for comparison."""
    tot = 0.0
    for delta, _, T in pairs:
        tot += float(((delta.float() - T) ** 2).mean())
    return tot / len(pairs)


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--pairs", type=int, default=2000)
    t.add_argument("--n", type=int, default=128)
    t.add_argument("--epochs", type=int, default=4)
    t.add_argument("--lr", type=float, default=1e-3)
    t.add_argument("--batch", type=int, default=8)
    t.add_argument("--seed", type=int, default=2000)
    t.add_argument("--out", default=os.path.join(WEIGHTS_DIR, "unet_128"))
    args = ap.parse_args()
    api.load()
    ctx = api.default_context()
    net = api.UNet(ctx)
    net.set_params(init_params(args.seed))
    t0 = time.time()
    pairs = make_pairs(args.pairs, args.n, args.seed, ctx)
    t_data = time.time() - t0
    held = pairs[-max(1, len(pairs) // 20):]
    train_set = pairs[: len(pairs) - len(held)]
    base = linear_loss(held)
    t1 = time.time()
    hist = train(net, train_set, args.epochs, args.lr, args.batch, args.seed)
    t_train = time.time() - t1
    held_loss = sum(net.loss_grad(d, T, *p) for d, p, T in held) / len(held)
    net.zero_grad()
    print(f"held-out loss {held_loss:.5f} (linear source {base:.5f}); data {t_data:.0f} s, training {t_train:.0f} s")
    save(net, args.out, {"trained_on": f"{len(train_set)} pairs at {args.n}^3 (seed {args.seed})",
                         "epochs": args.epochs, "loss_history": hist, "heldout_loss": held_loss,
                         "heldout_linear_loss": base, "data_seconds": t_data, "train_seconds": t_train})


if __name__ == "__main__":
    main()
