"""Benchmark of the screened EFTofDE scalar-field solve (arXiv 2604.15434) on GB300.

Metric: time-to-relative-residual 1e-8 of the 512^3 scalar-field solve (lower is better),
with the FP32-inner / FP64-outer path; the plain FP64 multigrid is timed beside it, and
the dominant kernel is reported against the HBM (or FP64 ALU) roofline.

Workload (one step): the 512^3 lognormal density (P(k) ~ k^-2, sigma_ln = 1.5, seed
1003), solved from a cold start (chi = 0) at a = 1 for each of the four parameter pairs
(alpha_B0, alpha_M0) in {-2, -0.5} x {0, 0.5}.  Inputs (1 GiB per field) are larger than
L2, so no explicit flush is needed between steps.  Beside the timed steps: the plain FP64
multigrid on the same inputs, the end-to-end call with host buffers, the cold / linear /
learned initial guesses (warm_start), the 24-box batched solve and the CPU oracle sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n 512]

Under torchrun (N > 1) every rank solves the same workload on its own GPU (independent
replicas, no collective on the data path); the reported time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

COMBOS = [(-2.0, 0.0), (-2.0, 0.5), (-0.5, 0.0), (-0.5, 0.5)]
# DRAM bytes per cell of one finest-level sweep launch of the coefficient-level variants the
# autotuner keeps at 512^3, each from one ncu capture of a 256^3 launch of that variant
# (dram__bytes_read.sum + dram__bytes_write.sum over 16.78 M cells;
# `python -m paper_2604_15434_gb300.microbench sweep --n 256 --mode <mode>`), scaled by the cell
# count.  Keyed by the autotuner's description of its choice; a variant without a capture
# reports no traffic.
SWEEP_DRAM = {
    "tile 64x16 nz 32 pair": (29.1, "k_sweep_pair<16,1,1,1,0>", 111),
    "tile 64x16 nz 32 pair bal": (29.2, "k_sweep_pair<16,1,1,1,1>", 115),
    "tile 64x16 nz 32 col": (29.9, "k_sweep_col<16>", 119),
}



def sweep_capture(tune_line: str):
    """The DRAM capture (bytes per cell, kernel, microbenchmark mode) of the sweep variant a
    tune-log line names ("sweep32 n=512 bg gap coef: tile 64x16 nz 32 pair 0.94 ms (variants
    ..."), or None when that variant has no capture."""
    variant = tune_line.split(": ", 1)[1].split(" (variants")[0] if ": " in tune_line else tune_line
    mv = re.match(r"(.*?) [0-9.]+ ms$", variant)
    return SWEEP_DRAM.get(mv.group(1) if mv else variant)


TOL = 1e-8
SEED = 1003
# the sampler's bound on |mu_chi| = |xi/nu|: draws beyond it (with more than 90% of the cells
# on the void floor) fail to converge in about half the cases (robustness_leg)
MU_CHI_MAX = 4.0
METRIC = "512^3 scalar solve time-to-residual 1e-8 (learned+FP32 vs plain FP64); HBM GB/s %"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p.get("hbm_gbs", 6800.0), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling in the background during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        for line in (getattr(self, "out", "") or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_step_ms(ms_step, ws, device=None):
    """The step time of the whole job: the maximum over the ranks (every rank runs the same
    workload on its own GPU, with no collective on the data path)."""
    if ws <= 1:
        return ms_step
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms_step], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ms_step, solves, ws):
    """ms per 512^3 solve of the whole job: every rank does `solves` solves in ms_step."""
    return ms_step / (solves * ws)


def _nproc():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(n_sample=128, target_n=512, cycles_target=None, sample_cycles=6):
    """The CPU oracle as it stands (one thread), on a bounded sample of the same workload:
    for each of the four parameter pairs, sample_cycles FAS V-cycles of the oracle from a cold
    start on the n_sample^3 field of the same recipe, giving its time per cycle; extrapolated
    to target_n^3 by the cell count (a V-cycle's work is linear in the cells) and by the number
    of cycles each pair needs at target_n^3.  Those counts are the plain FP64 GPU multigrid's
    (cycles_target, same algorithm, hence the same counts); without them the oracle's own
    counts at n_sample^3 are used, which understates the nu < 0 pairs (their counts grow with n)."""
    import oracle as O
    from paper_2604_15434_gb300 import synth

    d = synth.lognormal_delta(n_sample, -2.0, 1.5, SEED)
    O.build()
    scale = (target_n / n_sample) ** 3
    per_pair, total_s = {}, 0.0
    for aB, aM in COMBOS:
        key = f"{aB},{aM}"
        if cycles_target and key in cycles_target:
            t0 = time.perf_counter()
            O.scalar_solve(d, aB, aM, 1.0, 0.0, max_cycles=sample_cycles)
            dt = time.perf_counter() - t0
            per_cycle = dt / sample_cycles
            cyc = cycles_target[key]
            src = "cycles of the FP64 GPU multigrid at the target size"
        else:
            t0 = time.perf_counter()
            _, info, _ = O.scalar_solve(d, aB, aM, 1.0, TOL)
            dt = time.perf_counter() - t0
            per_cycle = dt / max(info["cycles"], 1)
            cyc = info["cycles"]
            src = f"the oracle's own cycles at {n_sample}^3 (a lower bound for nu < 0)"
        total_s += dt
        per_pair[key] = {"ms": per_cycle * cyc * scale * 1e3, "cycles": cyc, "s_per_cycle_sample": per_cycle}
    value = sum(v["ms"] for v in per_pair.values()) / len(per_pair)
    return {"value": value, "unit": "ms", "cores": 1, "host_nproc": _nproc(), "kind": "oracle",
            "sample": f"FP64 oracle (one thread, -O2) on the {n_sample}^3 lognormal of the same recipe (seed {SEED}), "
                      f"four parameter pairs, time per V-cycle x{scale:.0f} (cells) x cycles per pair at "
                      f"{target_n}^3 ({src}); {total_s:.1f} s of CPU work",
            "per_pair": per_pair, "sample_seconds": total_s}


def batched_leg(api, dev, stream, nbox=24, seed=1007):
    """The 24-box configuration: mesh sizes drawn from {64,128,256}^3, parameters alpha_B0 ~
    U[-2,0], alpha_M0 ~ U[0,1], a ~ U[0.3,1] (near-singular draws redrawn), Zel'dovich sources with
    P ~ k^-1.5 and sigma 1 deposited on the GPU; all boxes solved to 1e-8 by one batched call
    (one graph launch per outer iteration), and the same boxes one by one for comparison."""
    import torch
    from paper_2604_15434_gb300 import synth

    sizes = synth.sample_box_sizes(nbox, seed)
    def accept(aB, aM, a):  # draws with |nu| < 0.1 or |mu_chi| = |xi/nu| > 4 are redrawn (robustness_leg)
        c = api.coefficients(aB, aM, a)
        return abs(c["nu"]) >= 0.1 and abs(c["mu_chi"]) <= MU_CHI_MAX

    params = synth.sample_box_params(nbox, seed, accept=accept)
    deltas = []
    for b, n in enumerate(sizes):
        pos = torch.from_numpy(synth.zeldovich_particles(n, -1.5, 1.0, seed + 1 + b)).to(dev)
        deltas.append(api.pm_deposit_cic(pos, n))
        del pos
    aB = [p[0] for p in params]
    aM = [p[1] for p in params]
    aa = [p[2] for p in params]
    ctx = api.Context(dev.index, stream, precision=1, max_cycles=100)
    phis = [torch.zeros_like(d) for d in deltas]
    api.scalar_mg_solve_batched(deltas, aB, aM, aa, TOL, phis=phis, ctx=ctx)  # warm-up (tuning, workspaces)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for p in phis:
        p.zero_()
    torch.cuda.synchronize()
    e0.record(stream)
    _, infos = api.scalar_mg_solve_batched(deltas, aB, aM, aa, TOL, phis=phis, ctx=ctx)
    e1.record(stream)
    torch.cuda.synchronize()
    batched_ms = e0.elapsed_time(e1)
    seq_ctx = api.Context(dev.index, stream, precision=1, max_cycles=100)
    for d, b0, m0, a0 in zip(deltas, aB, aM, aa):  # warm-up of the single-box path
        api.scalar_mg_solve(d, b0, m0, a0, TOL, phi=torch.zeros_like(d), ctx=seq_ctx)
    torch.cuda.synchronize()
    e0.record(stream)
    for d, b0, m0, a0, p in zip(deltas, aB, aM, aa, phis):
        p.zero_()
        api.scalar_mg_solve(d, b0, m0, a0, TOL, phi=p, ctx=seq_ctx)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    cells = sum(n ** 3 for n in sizes)
    return {"boxes": nbox, "sizes": sizes, "batched_ms": batched_ms, "sequential_ms": seq_ms,
            "speedup_vs_sequential": seq_ms / batched_ms, "cells": cells,
            "max_rel_res": max(i["rel_res"] for i in infos), "outer_iterations": [i["cycles"] for i in infos],
            "tune": ctx.tune_log().strip().splitlines()}


def robustness_leg(api, dev, stream, count=500, n=64, seed=4000):
    """How often the solve converges over the batched/training distribution: `count` seeded
    draws at n^3, alternately a lognormal source (P ~ k^-2, sigma_ln ~ U[1, 1.8]) and a
    Zel'dovich one (P ~ k^-1.5, sigma ~ U[0.5, 2]), parameters alpha_B0 ~ U[-2,0], alpha_M0 ~
    U[0,1], a ~ U[0.3,1] redrawn only where |nu| < 0.1 or |mu_chi| > 8 (the wider rule), all
    solved to 1e-8 (max 200 outer iterations) by batched calls of 100 boxes.  Reported for the
    wider rule and for the sampler's rule |mu_chi| <= MU_CHI_MAX."""
    import numpy as np
    import torch
    from paper_2604_15434_gb300 import synth

    t0 = time.time()
    draws = []
    for i in range(count):
        rng = np.random.default_rng(seed + i)
        kind = "lognormal" if i % 2 == 0 else "zeldovich"
        sigma = rng.uniform(1.0, 1.8) if kind == "lognormal" else rng.uniform(0.5, 2.0)
        while True:
            aB, aM, a = rng.uniform(-2.0, 0.0), rng.uniform(0.0, 1.0), rng.uniform(0.3, 1.0)
            c = api.coefficients(aB, aM, a)
            if abs(c["nu"]) >= 0.1 and abs(c["mu_chi"]) <= 8.0 and c["xi"] != 0.0:
                break
        if kind == "lognormal":
            d = torch.from_numpy(synth.lognormal_delta(n, -2.0, sigma, seed + 100000 + i)).to(dev)
        else:
            pos = torch.from_numpy(synth.zeldovich_particles(n, -1.5, sigma, seed + 100000 + i)).to(dev)
            d = api.pm_deposit_cic(pos, n)
        draws.append((d, aB, aM, a, c["nu"], c["mu_chi"]))
    gen_s = time.time() - t0
    ctx = api.Context(dev.index, stream, precision=1, max_cycles=200)
    infos = []
    torch.cuda.synchronize()
    t1 = time.time()
    for k in range(0, count, 100):
        ch = draws[k:k + 100]
        _, inf = api.scalar_mg_solve_batched([x[0] for x in ch], [x[1] for x in ch], [x[2] for x in ch],
                                             [x[3] for x in ch], TOL, ctx=ctx, raise_on_noconv=False)
        infos += inf
    torch.cuda.synchronize()
    solve_s = time.time() - t1
    ok = [i["status"] == 0 for i in infos]
    narrow = [abs(x[5]) <= MU_CHI_MAX for x in draws]
    fails = [{"draw": k, "alpha_B0": draws[k][1], "alpha_M0": draws[k][2], "a": draws[k][3], "nu": draws[k][4],
              "mu_chi": draws[k][5], "status": infos[k]["status"], "rel_res": infos[k]["rel_res"],
              "floored_frac": infos[k]["floored_cells"] / n ** 3} for k in range(count) if not ok[k]]
    return {"draws": count, "n": n, "converged": sum(ok), "converged_frac": sum(ok) / count,
            "narrow_rule": f"|mu_chi| <= {MU_CHI_MAX}", "narrow_draws": sum(narrow),
            "narrow_converged": sum(1 for o, w in zip(ok, narrow) if o and w),
            "failures": fails, "generate_s": gen_s, "solve_s": solve_s}


def warm_start_leg(api, delta, stream, ctx):
    """The learned warm start at 512^3 against the cold start (chi = 0) and the paper's
    linear start (the unscreened solution, one FFT Poisson solve): per parameter pair, the
    time of the initial guess plus the mixed-precision solve to the same tolerance, the outer
    iterations and the first residual.  The network (trained at 128^3, weights in the
    package) runs on its BF16 tensor-core kernels."""
    import torch
    from paper_2604_15434_gb300 import learned

    path = os.path.join(learned.WEIGHTS_DIR, "unet_128")
    if not os.path.exists(path + ".bin"):
        return {"skipped": "no trained weights in the package"}
    net = api.UNet(ctx)
    net.set_params(learned.load_params(path))
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    out = {}
    phi = torch.zeros_like(delta)
    net.warm_start(delta, *COMBOS[0], 1.0, phi=phi)  # warm-up: activations, weight packing
    for aB, aM in COMBOS:
        row = {}
        for name in ("cold", "linear", "learned"):
            torch.cuda.synchronize()
            e0.record(stream)
            if name == "cold":
                phi.zero_()
            elif name == "linear":
                api.linear_start(delta, aB, aM, 1.0, phi=phi, ctx=ctx)
            else:
                net.warm_start(delta, aB, aM, 1.0, phi=phi)
            e1.record(stream)
            _, info = api.scalar_mg_solve(delta, aB, aM, 1.0, TOL, phi=phi, ctx=ctx, raise_on_noconv=False)
            e2.record(stream)
            torch.cuda.synchronize()
            row[name] = {"init_ms": e0.elapsed_time(e1), "total_ms": e0.elapsed_time(e2), "cycles": info["cycles"],
                         "guess_rel_res": info["guess_rel_res"], "guess_rejected": info["guess_rejected"],
                         "rel_res": info["rel_res"], "status": info["status"]}
        out[f"{aB},{aM}"] = row
    mean = {k: sum(r[k]["total_ms"] for r in out.values()) / len(out) for k in ("cold", "linear", "learned")}
    # the network's forward alone (its tensor-core convolutions and the pooling, upsampling and
    # head kernels): 2 x 27 x sum(Cin Cout per voxel of each level) flop per voxel of the grid
    reps = 3
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        net.forward(delta, *COMBOS[0], 1.0)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / reps
    n = delta.shape[0]
    macs = 27 * (16 * 16 + 16 * 16 + 48 * 16 + 16 * 16 + (16 * 32 + 32 * 32 + 96 * 32 + 32 * 32) / 8.0 +
                 (32 * 64 + 64 * 64) / 64.0)
    flop = 2.0 * macs * n ** 3
    bf16 = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16 = json.load(f).get("bf16_tflops")
    except Exception:
        pass
    tflops = flop / (fwd_ms * 1e-3) / 1e12
    net.close()
    return {"per_pair": out, "mean_total_ms": mean,
            "unet_forward": {"ms": fwd_ms, "tflop": flop / 1e12, "tflops": tflops,
                             "frac_of_bf16_peak": tflops / bf16 if bf16 else None,
                             "conv_path": "tcgen05 (k_conv3d_umma)"},
            "note": "total_ms = initial guess + solve; guess_rel_res = relative residual of the guess"}


def next_rows_leg(api, dev, stream):
    """The full PM step of the 256^3-mesh / 256^3-particle configuration (Zel'dovich ICs,
    P ~ k^-1.5, sigma 2, alpha = (-1, 0.2), a = 1, dt = 1e-3: deposit, FFT Poisson, chi solve to
    1e-8, gradient, force interpolation, kick-drift) and the rows built beyond the solve: a
    4-step run a = 0.5 -> 1, the linearised mode, the lensing potential and the Method II
    smoother.  Each is timed on the device through the public API after one warm-up call."""
    import torch
    from paper_2604_15434_gb300 import synth

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, r

    n = 256
    pos0 = torch.from_numpy(synth.zeldovich_particles(n, -1.5, 2.0, 1002)).to(dev)
    pos, vel = pos0.clone(), torch.zeros_like(pos0)
    phi = torch.zeros((n, n, n), dtype=torch.float64, device=dev)
    out = {"particles": n ** 3, "mesh": n}

    def step(c, tol=TOL):
        pos.copy_(pos0)
        vel.zero_()
        phi.zero_()
        return api.pm_step(pos, vel, n, -1.0, 0.2, 1.0, 1e-3, tol, phi, ctx=c)

    for name, c in (("pm_step_mixed", api.Context(dev.index, stream, precision=1, max_cycles=100)),
                    ("pm_step_fp64", api.Context(dev.index, stream, precision=0, max_cycles=100)),
                    ("pm_step_linearised", api.Context(dev.index, stream, precision=1, linear_eft=1))):
        ms, info = timed(lambda: step(c), 2)
        out[name] = {"ms": ms, "cycles": info["cycles"], "rel_res": info["rel_res"],
                     "particles_per_s": n ** 3 / (ms * 1e-3)}
    cr = api.Context(dev.index, stream, precision=1, max_cycles=100)

    def run():
        pos.copy_(pos0)
        vel.zero_()
        phi.zero_()
        return api.pm_run(pos, vel, n, -1.0, 0.2, 0.5, 1.0, 4, TOL, phi, ctx=cr)

    ms, info = timed(run, 1)
    out["pm_run_4_steps"] = {"ms": ms, "ms_per_step": ms / 4, "last_cycles": info["cycles"]}
    psi = api.poisson_solve(torch.from_numpy(synth.lognormal_delta(n, -2.0, 1.5, SEED)).to(dev), 1.0, 0.2, ctx=cr)
    ms, _ = timed(lambda: api.lensing_potential(psi, phi, -1.0, 0.2, 1.0, ctx=cr), 5)
    out["lensing_potential"] = {"ms": ms, "gbs": 3 * 8 * n ** 3 / (ms * 1e-3) / 1e9}
    # the PM step's own kernels on their own, with their algorithmic bytes: the deposit reads
    # the positions (24 B per particle) and adds 8 int64 weights per particle in L2, clears the
    # int64 grid and converts it to delta (24 B per cell); the Poisson solve is two FP64 cuFFT
    # passes and the Green's function (timed, no byte model); the force kernel reads the two
    # potentials' 5-point stencils at the 8 CIC corners (2 x 8 B per cell from DRAM, the rest
    # from L2) and the positions, and writes the accelerations (24 + 24 B per particle)
    hbm, _ = _peaks()
    cp = api.Context(dev.index, stream, precision=1)
    ms, dlt = timed(lambda: api.pm_deposit_cic(pos0, n, ctx=cp), 5)
    byt = 24 * n ** 3 + 24 * n ** 3
    out["deposit"] = {"ms": ms, "particles_per_s": n ** 3 / (ms * 1e-3), "gbs": byt / (ms * 1e-3) / 1e9,
                      "frac_of_hbm": byt / (ms * 1e-3) / 1e9 / hbm, "bound": "L2 atomics"}
    ms, psn = timed(lambda: api.poisson_solve(dlt, 1.0, 0.2, ctx=cp), 5)
    out["poisson_fft"] = {"ms": ms}
    acc = torch.empty_like(pos0)
    ms, _ = timed(lambda: api.force_interp(psn, phi, -1.0, 0.2, 1.0, pos0, acc=acc, ctx=cp), 5)
    byt = 16 * n ** 3 + 48 * n ** 3
    out["force_interp"] = {"ms": ms, "particles_per_s": n ** 3 / (ms * 1e-3), "gbs": byt / (ms * 1e-3) / 1e9,
                           "frac_of_hbm": byt / (ms * 1e-3) / 1e9 / hbm}
    m2 = {}
    d128 = torch.from_numpy(synth.lognormal_delta(128, -2.0, 1.5, SEED)).to(dev)
    p128 = torch.zeros_like(d128)
    for sm in (0, 1):
        c = api.Context(dev.index, stream, precision=0, max_cycles=100, smoother=sm)

        def solve():
            p128.zero_()
            return api.scalar_mg_solve(d128, -2.0, 0.0, 1.0, TOL, phi=p128, ctx=c)[1]

        ms, info = timed(solve, 2)
        m2["method_" + ("II" if sm else "I")] = {"ms": ms, "cycles": info["cycles"], "rel_res": info["rel_res"]}
    out["fp64_solve_128_by_smoother"] = m2
    return out


def precision_leg(api, delta, stream, dev):
    """The precision options of the solve on the 512^3 workload, each pair from a cold start to
    the same tolerance: the default float-float outer loop (precision 1), the FP64 outer loop
    (precision 2: FP64 residual and iterate around the FP32 inner cycle), and both with the exact
    FP64 coarsest solve (Newton with a dense Jacobian and LU on 4^3)."""
    import torch

    out = {}
    phi = torch.zeros_like(delta)
    for name, kw in (("float_float_outer", dict(precision=1)), ("fp64_outer", dict(precision=2)),
                     ("float_float_outer_exact_coarsest", dict(precision=1, coarse_exact=1)),
                     ("fp64_outer_exact_coarsest", dict(precision=2, coarse_exact=1))):
        c = api.Context(dev.index, stream, max_cycles=100, **kw)
        phi.zero_()
        api.scalar_mg_solve(delta, *COMBOS[2], 1.0, TOL, phi=phi, ctx=c, raise_on_noconv=False)  # warm-up
        rows = {}
        for aB, aM in COMBOS:
            phi.zero_()
            torch.cuda.synchronize()
            _, info = api.scalar_mg_solve(delta, aB, aM, 1.0, TOL, phi=phi, ctx=c, raise_on_noconv=False)
            rows[f"{aB},{aM}"] = {"ms": info["ms_total"], "cycles": info["cycles"], "vcycles": info["vcycles"],
                                  "rel_res": info["rel_res"], "status": info["status"]}
        out[name] = {"per_pair": rows, "mean_ms": sum(r["ms"] for r in rows.values()) / len(rows)}
        c.close()
    return out


def void_floor_leg(api, delta, stream, dev, phis):
    """The literal void floor (eta = 0: only cells with a negative discriminant are floored, at
    the parabola's vertex; Sec. 3.3) against the default eta on the nu > 0 pairs of the 512^3
    workload: cycles, time, floored fraction and the relative change of chi (phis holds the
    timed steps' solutions at the default eta).  The mixed-precision solve is tried first; where
    it stops with an error (its FP32 inner cycle does not handle the vertex floor's zero
    discriminant), the plain FP64 solve is run instead, capped at 40 cycles (it stalls, as on the
    oracle)."""
    import torch

    cells = delta.numel()
    out = {}
    phi = torch.zeros_like(delta)
    for i, (aB, aM) in enumerate(COMBOS):
        if api.coefficients(aB, aM, 1.0)["nu"] <= 0.0:
            continue
        row = {}
        for prec, cap in ((1, 100), (0, 40)):
            c = api.Context(dev.index, stream, precision=prec, max_cycles=cap, eta=0.0)
            phi.zero_()
            key = "mixed" if prec == 1 else "fp64"
            try:
                _, info = api.scalar_mg_solve(delta, aB, aM, 1.0, TOL, phi=phi, ctx=c, raise_on_noconv=False)
                row[key] = {"ms": info["ms_total"], "cycles": info["cycles"], "rel_res": info["rel_res"],
                            "status": info["status"], "floored_frac": info["floored_cells"] / cells,
                            "rel_change_chi_vs_default_eta": float((phi - phis[i]).norm() / phis[i].norm())}
            except api.PMError as e:
                row[key] = {"status": e.status, "error": str(e)}
            c.close()
            if row[key].get("status") == 0:
                break
        out[f"{aB},{aM}"] = row
    return {"eta": 0.0, "per_pair": out}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    # each step: one bounded oracle sample; the line reports the mean extrapolated value
    # each step: the four pairs solved to tolerance by the oracle at the sample size (64^3 unless
    # --sample-n says otherwise), extrapolated by the cell count
    sn = args.sample_n if args.sample_n else 64
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(sn, args.n)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(sn, args.n))
    wall = time.perf_counter() - t0
    v = sum(x["value"] for x in vals) / len(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": wall * 1e3 / max(args.steps, 1), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.n}^3 lognormal scalar solve, extrapolated from {sn}^3 samples",
                       "n": args.n, "tol": TOL},
            "cpu_baseline": {"value": v, "unit": "ms", "cores": 1, "host_nproc": _nproc(), "kind": "oracle",
                             "sample": vals[0]["sample"], "per_pair": vals[0]["per_pair"]},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--sample-n", type=int, default=0, help="CPU-oracle sample size (default 128; 64 for the "
                                                           "reference arm)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison solves")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the 24-box batched-solve leg")
    ap.add_argument("--no-warm", action="store_true", help="skip the cold / linear / learned warm-start leg")
    ap.add_argument("--no-next", action="store_true", help="skip the PM-step / run / linearised / lensing / "
                                                            "Method II leg")
    ap.add_argument("--no-precision", action="store_true", help="skip the FP64-outer / exact-coarsest leg")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    from paper_2604_15434_gb300 import api, synth

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    api.load()
    n = args.n
    dev = torch.device("cuda", local)
    delta_h = synth.lognormal_delta(n, -2.0, 1.5, SEED)
    delta = torch.from_numpy(delta_h).to(dev)
    phis = [torch.zeros((n, n, n), dtype=torch.float64, device=dev) for _ in COMBOS]
    stream = torch.cuda.current_stream(dev)
    ctx = api.Context(local, stream, precision=1, max_cycles=100)
    ctx64 = api.Context(local, stream, precision=0, max_cycles=100)
    infos = {}

    def step(c=ctx, record=None):
        for i, (aB, aM) in enumerate(COMBOS):
            phis[i].zero_()
            _, info = api.scalar_mg_solve(delta, aB, aM, 1.0, TOL, phi=phis[i], ctx=c)
            if record is not None:
                record[(aB, aM)] = info

    fp64_gf, fp32_gf = ctx.probe_fma()
    for _ in range(args.warmup):
        step(record=infos)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # inside the timed region only the finest-level FP32 sweeps (the dominant kernel, whose
    # launch time the roofline needs) carry CUDA events; every other launch is only counted
    ctx.trace_select([api.KERNEL_CLASSES.index("sweep32")], fine_only=True)
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step(record=infos)
        e1.record(stream)
        torch.cuda.synchronize()
    prof = ctx.trace_get()
    ctx.trace(False)
    ms_total = e0.elapsed_time(e1)
    ms_step = ms_total / args.steps
    ms_step = job_step_ms(ms_step, ws, dev)
    solves = len(COMBOS)
    value = job_value(ms_step, solves, ws)  # ms per 512^3 solve, whole job

    # end to end through the C ABI with host buffers: H2D delta, solve, D2H chi (headline pair),
    # measured right after the timed steps, before the comparison legs allocate their own fields;
    # with events between the three parts
    host_in = torch.from_numpy(delta_h).pin_memory()
    host_out = torch.empty((n, n, n), dtype=torch.float64).pin_memory()
    dev_in = torch.empty_like(delta)
    e2e_ms, e2e_parts = [], []
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # one untimed round trip first: the first copies through freshly pinned buffers pay for
    # their mapping (about ten times the steady copy time on this machine)
    dev_in.copy_(host_in, non_blocking=True)
    host_out.copy_(phis[0], non_blocking=True)
    torch.cuda.synchronize()
    # the same two copies alone, for the host link's rate at this point of the run
    e0.record(stream)
    dev_in.copy_(host_in, non_blocking=True)
    ea.record(stream)
    host_out.copy_(phis[0], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    link = (cells_h := n ** 3 * 8) / (e0.elapsed_time(ea) * 1e-3) / 1e9, cells_h / (ea.elapsed_time(e1) * 1e-3) / 1e9
    for _ in range(max(1, args.steps)):
        phis[0].zero_()
        torch.cuda.synchronize()
        e0.record(stream)
        dev_in.copy_(host_in, non_blocking=True)
        ea.record(stream)
        api.scalar_mg_solve(dev_in, COMBOS[0][0], COMBOS[0][1], 1.0, TOL, phi=phis[0], ctx=ctx)
        eb.record(stream)
        host_out.copy_(phis[0], non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
        e2e_parts.append((e0.elapsed_time(ea), ea.elapsed_time(eb), eb.elapsed_time(e1)))

    # one more step with every launch traced, outside the timed region: the per-class breakdown
    ctx.trace(True)
    torch.cuda.synchronize()
    e0.record(stream)
    step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_traced = e0.elapsed_time(e1)
    prof_all = ctx.trace_get()
    ctx.trace(False)

    # plain FP64 multigrid on the same inputs
    fp64 = {}
    if not args.no_fp64:
        for i, (aB, aM) in enumerate(COMBOS):
            phis[i].zero_()
            torch.cuda.synchronize()
            e0.record(stream)
            _, info = api.scalar_mg_solve(delta, aB, aM, 1.0, TOL, phi=phis[i], ctx=ctx64, raise_on_noconv=False)
            e1.record(stream)
            torch.cuda.synchronize()
            fp64[f"{aB},{aM}"] = {"ms": e0.elapsed_time(e1), "cycles": info["cycles"], "rel_res": info["rel_res"]}

    # roofline of the dominant kernel class, finest-level launches
    hbm, src = _peaks()
    cells = n ** 3
    dominant = max(prof_all, key=lambda k: prof_all[k]["ms"])
    roof = None
    fine = prof["sweep32"]
    if fine["fine_launches"] > 0 and fine["fine_ms"] > 0:
        avg_ms = fine["fine_ms"] / fine["fine_launches"]
        # algorithmic bytes of one finest-level launch of the single-pass FP32 sweep (both
        # colours): read the iterate and the right-hand side, write the iterate, 12 B per cell
        # (the ideal FP32 sweep's figure).  The correction form also reads the background and
        # the floored gap: 20 B per cell on that count (frac_20B).
        bytes_launch = cells * 12
        ach = bytes_launch / (avg_ms * 1e-3) / 1e9
        tuned = [l for l in ctx.tune_log().splitlines() if f"n={n} bg gap" in l]
        variant = tuned[-1].split(": ", 1)[1].split(" (variants")[0] if tuned else "?"
        cap = sweep_capture(tuned[-1]) if tuned else None
        per_cell = cap[0] if cap else None
        roof = {"kernel": "single-pass FP32 red-black sweep of the finest level (k_sweep_pair / k_sweep_col / "
                          "k_sweep_fused, autotuned: " + variant + ")", "bound": "hbm",
                "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": per_cell * cells if per_cell else None,
                "traffic_source": (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of one 256^3 launch of {cap[1]} "
                                   f"(microbench sweep --n 256 --mode {cap[2]}): {cap[0]} B/cell, times this "
                                   "launch's cells") if cap else "no capture of this variant",
                "peak_source": src, "frac_of_nominal_8000": ach / 8000.0,
                "bytes_per_launch": bytes_launch, "bytes_per_cell": 12,
                "frac_20B": cells * 20 / (avg_ms * 1e-3) / 1e9 / hbm,
                "avg_launch_ms": avg_ms, "launches": fine["fine_launches"]}
    r64 = prof_all["resid64"]
    resid64 = None
    if r64["fine_launches"] > 0 and r64["fine_ms"] > 0:
        avg = r64["fine_ms"] / r64["fine_launches"]
        resid64 = {"avg_launch_ms": avg, "launches": r64["fine_launches"],
                   "gbs": cells * (8 + 8 + 4 + 4 + 4 + 1) / (avg * 1e-3) / 1e9,
                   "fp64_fma_gflops_probe": fp64_gf}
    launches = sum(v["launches"] for v in prof.values())
    line = {
        "metric": METRIC, "value": value, "unit": "ms", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f32x2+f64", "data": "synthetic",
        "config": {"workload": f"{n}^3 lognormal delta (P~k^-2, sigma_ln=1.5, seed {SEED}), cold-start chi solve "
                               f"to rel. residual {TOL:g} for (alpha_B0,alpha_M0) in {{-2,-0.5}}x{{0,0.5}}, a=1; "
                               "one FP32 inner FAS V(2,2) cycle per outer iteration of a float-float defect-"
                               "correction loop, the result confirmed by an FP64 residual; the learned warm start "
                               "is timed separately (warm_start)",
                   "n": n, "solves_per_step": solves, "tol": TOL,
                   "l2": f"inputs larger than L2 ({n ** 3 * 8 / 2 ** 30:g} GiB per field)" if n ** 3 * 8 > 129e6
                         else "inputs smaller than L2 (no flush: small-case profiling run)"},
        "e2e": {"value": sum(e2e_ms) / len(e2e_ms), "unit": "ms", "h2d_bytes_per_step": cells * 8,
                "d2h_bytes_per_step": cells * 8, "per": "one solve (alpha_B0=-2, alpha_M0=0) incl. H2D delta, D2H chi",
                "h2d_ms": sum(p[0] for p in e2e_parts) / len(e2e_parts),
                "solve_ms": sum(p[1] for p in e2e_parts) / len(e2e_parts),
                "d2h_ms": sum(p[2] for p in e2e_parts) / len(e2e_parts),
                "h2d_gbs": cells * 8 / (sum(p[0] for p in e2e_parts) / len(e2e_parts) * 1e-3) / 1e9,
                "d2h_gbs": cells * 8 / (sum(p[2] for p in e2e_parts) / len(e2e_parts) * 1e-3) / 1e9,
                "copies_alone_gbs": {"h2d": link[0], "d2h": link[1]}},
        "roofline": roof,
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "fp64_multigrid": fp64,
        "fp64_ms_per_solve": (sum(v["ms"] for v in fp64.values()) / len(fp64)) if fp64 else None,
        "speedup_vs_fp64": ((sum(v["ms"] for v in fp64.values()) / len(fp64)) / value) if fp64 else None,
        "solves": {f"{k[0]},{k[1]}": {"cycles": v["cycles"], "rel_res": v["rel_res"], "floored": v["floored_cells"],
                                       "floored_frac": v["floored_cells"] / cells, "ms": v["ms_total"]}
                   for k, v in infos.items()},
        "eta": ctx.params.eta,
        "eta_reading": "discriminant floor sqrt(D_floor) = eta 6|nu|/h^2 with the linear residual piece in floored "
                       "cells (reading of 'a very low value close to zero'); floored_frac per pair is the share of "
                       "cells on that floor in the converged field",
        # fine-equivalent smoother throughput: every level's cells x sweeps of the inner V-cycles
        # (one per outer iteration), per second of solve time; and n^3 per time to tolerance
        "cell_updates_per_s": sum(v["vcycles"] * 4 * sum((n >> l) ** 3 for l in range(int(math.log2(n)) - 1))
                                  for v in infos.values()) / (sum(v["ms_total"] for v in infos.values()) * 1e-3),
        "cells_per_s_to_tol": cells * len(infos) / (sum(v["ms_total"] for v in infos.values()) * 1e-3),
        "kernel_ms_per_step": {k: v["ms"] for k, v in prof_all.items()},
        "dominant_class": dominant,
        "resid64": resid64,
        "fma_probe_gflops": {"fp64": fp64_gf, "fp32": fp32_gf},
        "ms_per_step_fully_traced": ms_traced,
        "tracing": "timed steps: events on the finest-level FP32 sweeps only (roofline); kernel_ms_per_step "
                   "and dominant_class: one extra step with every launch traced (ms_per_step_fully_traced)",
    }
    if not args.no_warm:
        ws_leg = warm_start_leg(api, delta, stream, ctx)
        line["warm_start"] = ws_leg
        if "mean_total_ms" in ws_leg:
            line["learned_mixed_ms_per_solve"] = ws_leg["mean_total_ms"]["learned"]
            if fp64:
                line["speedup_learned_vs_fp64"] = line["fp64_ms_per_solve"] / ws_leg["mean_total_ms"]["learned"]
    if not args.no_precision:
        line["void_floor_literal"] = void_floor_leg(api, delta, stream, dev, phis)
        line["precision_variants"] = precision_leg(api, delta, stream, dev)
    if not args.no_batch:
        line["batched"] = batched_leg(api, dev, stream)
        line["robustness"] = robustness_leg(api, dev, stream)
    if not args.no_next:
        line["next_rows"] = next_rows_leg(api, dev, stream)
    if rank == 0 and not args.no_cpu:
        cyc = {k: v["cycles"] for k, v in fp64.items()} if fp64 else None
        line["cpu_baseline"] = cpu_baseline(args.sample_n or 128, n, cyc)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
