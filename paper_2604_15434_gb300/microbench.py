"""Kernel microbenchmarks through the C ABI, for timing and profiling single kernels.

    python -m paper_2604_15434_gb300.microbench sweep --n 256 --mode 115
    python -m paper_2604_15434_gb300.microbench unet --n 256 --path 1
    python -m paper_2604_15434_gb300.microbench pmstep --n 256

``sweep`` runs the finest-level FP32 sweep (pm_mg_sweep_f32) on seeded inputs of the
benchmark recipe: a lognormal source (P ~ k^-2, sigma_ln 1.5) for the pair (-0.5, 0), a
random correction and background, and a floored gap around L_sat.  ``--mode`` selects the
kernel as pm_mg_sweep_f32 documents (100 + k: tile variant k - 1 with the background
through its BF16 coefficients).  ``unet`` runs the warm-start network's forward pass (the
packaged weights when present, else a seeded initialisation) on a lognormal field.
``pmstep`` runs the particle-mesh step of the 256^3-mesh configuration (n^3 Zel'dovich
particles, P ~ k^-1.5, sigma 2, (alpha_B0, alpha_M0) = (-1, 0.2), a = 1, dt = 1e-3, mixed
precision, chi to 1e-8).  Each prints one JSON line per repetition with the CUDA-event time in
milliseconds.
"""
from __future__ import annotations

import argparse
import json
import os


def _sweep(args):
    import numpy as np
    import torch

    from . import api, synth

    n = args.n
    rng = np.random.default_rng(1)
    c = api.coefficients(-0.5, 0.0, 1.0)
    d = synth.lognormal_delta(n, -2.0, 1.5, 7)
    dev = torch.device("cuda", 0)
    f = torch.from_numpy(c["src"] * d).float().to(dev)
    u = torch.from_numpy(0.5 * rng.standard_normal((n, n, n)) / n ** 2).float().to(dev)
    bg = torch.from_numpy(2.0 * rng.standard_normal((n, n, n)) / n ** 2).float().to(dev)
    lsat = 0.75 * c["nu"] * (1 - 0.35) / c["kappa"]
    gap = torch.from_numpy(lsat * (1.0 + 0.5 * rng.standard_normal((n, n, n)))).float().to(dev)
    ctx = api.Context()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for rep in range(args.reps):
        x = u.clone()
        torch.cuda.synchronize()
        e0.record()
        api.pm_mg_sweep_f32(x, f, 0.01, c["nu"], c["kappa"], 0.35, mode=args.mode, bg=bg, gap=gap, ctx=ctx)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"kernel": "sweep", "n": n, "mode": args.mode, "rep": rep, "ms": e0.elapsed_time(e1)}),
              flush=True)


def _unet(args):
    import numpy as np
    import torch

    from . import api, learned

    n = args.n
    dev = torch.device("cuda", 0)
    path = os.path.join(learned.WEIGHTS_DIR, "unet_128")
    net = api.UNet()
    net.set_conv_path(args.path)
    if os.path.exists(path + ".bin"):
        net.set_params(learned.load_params(path))
    else:
        net.set_params(np.random.default_rng(5).standard_normal(net.num_params).astype(np.float32) * 0.05)
    g = torch.Generator(device=dev)
    g.manual_seed(3)
    d = (torch.randn((n, n, n), generator=g, device=dev, dtype=torch.float64) * 0.8).exp() - 1.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for rep in range(args.reps):
        torch.cuda.synchronize()
        e0.record()
        net.forward(d, -1.0, 0.2, 1.0)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"kernel": "unet_forward", "n": n, "path": args.path, "rep": rep,
                          "ms": e0.elapsed_time(e1)}), flush=True)
    net.close()


def _pmstep(args):
    import torch

    from . import api, synth

    n = args.n
    dev = torch.device("cuda", 0)
    pos0 = torch.from_numpy(synth.zeldovich_particles(n, -1.5, 2.0, 1002)).to(dev)
    pos, vel = pos0.clone(), torch.zeros_like(pos0)
    phi = torch.zeros((n, n, n), dtype=torch.float64, device=dev)
    ctx = api.Context(precision=1, max_cycles=100)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for rep in range(args.reps):
        pos.copy_(pos0)
        vel.zero_()
        phi.zero_()
        torch.cuda.synchronize()
        e0.record()
        info = api.pm_step(pos, vel, n, -1.0, 0.2, 1.0, 1e-3, 1e-8, phi, ctx=ctx)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"kernel": "pm_step", "n": n, "rep": rep, "ms": e0.elapsed_time(e1),
                          "cycles": info["cycles"]}), flush=True)
    print(json.dumps({"tune": ctx.tune_log().strip().splitlines()}), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    s = sub.add_parser("sweep")
    s.add_argument("--n", type=int, default=256)
    s.add_argument("--mode", type=int, default=115)
    s.add_argument("--reps", type=int, default=3)
    u = sub.add_parser("unet")
    u.add_argument("--n", type=int, default=256)
    u.add_argument("--path", type=int, default=1)
    u.add_argument("--reps", type=int, default=3)
    m = sub.add_parser("pmstep")
    m.add_argument("--n", type=int, default=256)
    m.add_argument("--reps", type=int, default=2)
    args = ap.parse_args(argv)
    {"sweep": _sweep, "unet": _unet, "pmstep": _pmstep}[args.cmd](args)


if __name__ == "__main__":
    main()
