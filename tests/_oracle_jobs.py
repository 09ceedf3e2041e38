"""Oracle reference computations for the large parity tests, run in worker processes.

Each function is self-contained (imports inside), so a process pool started with the
"spawn" method can run several of these slow single-threaded FP64 computations at once
while the GPU tests wait for them.  Nothing here touches the GPU.
"""
from __future__ import annotations

import numpy as np


def _accept(aB, aM, a):
    import oracle as O

    c = O.coefficients(aB, aM, a)
    return abs(c["nu"]) >= 0.1 and abs(c["mu_chi"]) <= 4.0


def lognormal_solve(n, aB0, aM0, tol, seed=1003, eta=None):
    """The oracle's chi for the benchmark recipe (lognormal, P ~ k^-2, sigma_ln 1.5) at a = 1."""
    import oracle as O
    from paper_2604_15434_gb300 import synth

    d = synth.lognormal_delta(n, -2.0, 1.5, seed)
    kw = {} if eta is None else {"eta": eta}
    chi, info, st = O.scalar_solve(d, aB0, aM0, 1.0, tol, **kw)
    return {"chi": chi, "cycles": info["cycles"], "rel_res": info["rel_res"], "status": st,
            "lambda": info["lambda"], "sat_cells": info["sat_cells"]}


def pm_step_c2(n, aB0, aM0, dt, tol, sample):
    """One oracle PM step of the Zel'dovich 256^3 configuration (P ~ k^-1.5, sigma 2, seed 1002);
    returns chi, the particle accelerations and the updated state on a particle sample."""
    import oracle as O
    from paper_2604_15434_gb300 import synth

    pos = synth.zeldovich_particles(n, -1.5, 2.0, 1002)
    out = O.pm_step(pos, np.zeros_like(pos), n, aB0, aM0, 1.0, dt, tol)
    s = np.asarray(sample)
    return {"chi": out["chi"], "acc": out["acc"][:, s], "pos": out["pos"][:, s], "vel": out["vel"][:, s],
            "status": out["status"], "cycles": out["info"]["cycles"]}


def box_set(sizes, seed, tol):
    """Mixed-size boxes of Zel'dovich sources (P ~ k^-1.5, sigma 1) with parameters drawn as for the
    batched configuration (near-singular draws redrawn); the oracle's delta and chi of each."""
    import oracle as O
    from paper_2604_15434_gb300 import synth

    params = synth.sample_box_params(len(sizes), seed, accept=_accept)
    out = []
    for b, (n, (aB, aM, a, _)) in enumerate(zip(sizes, params)):
        pos = synth.zeldovich_particles(n, -1.5, 1.0, seed + b)
        d = O.density(O.deposit_cic(pos, n), pos.shape[1])
        chi, info, st = O.scalar_solve(d, aB, aM, a, tol)
        out.append({"delta": d, "aB0": aB, "aM0": aM, "a": a, "chi": chi, "status": st,
                    "cycles": info["cycles"]})
    return out
