"""Pins of the FP64 reference of the warm-start network (CPU).

The tap convention is fixed by a closed form (a single-tap kernel shifts the field), the
hand-written backward pass by central finite differences of the loss, and the training
target by the linear limit (T = delta when the screening term is off)."""
import numpy as np
import pytest

import oracle as O
from oracle import unet as U


def test_single_tap_convolution_is_a_shift():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((8, 8, 8, 2))
    W = np.zeros((27, 2, 2))
    t = (0 + 1) * 9 + (0 + 1) * 3 + (1 + 1)  # (dz, dy, dx) = (0, 0, +1)
    W[t] = np.eye(2)
    y = U.conv(x, W, np.zeros(2))
    assert np.array_equal(y, np.roll(x, -1, axis=2))  # y[z,y,x] = x[z,y,x+1]
    t = (-1 + 1) * 9 + (1 + 1) * 3 + (0 + 1)  # (dz, dy, dx) = (-1, +1, 0)
    W[:] = 0
    W[t] = np.eye(2)
    assert np.array_equal(U.conv(x, W, np.zeros(2)), np.roll(x, (1, -1), axis=(0, 1)))


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    n = 8
    p = U.init_params(3)
    p[-1] = 0.2
    delta = np.exp(rng.standard_normal((n, n, n))) - 1.0
    target = rng.standard_normal((n, n, n))
    loss, g = U.loss_grad(p, delta, target, -0.7, 0.3, 0.8)
    offs = np.cumsum([0] + [27 * ci * co + co for ci, co in U.CONVS])
    idx = [int(offs[k] + rng.integers(0, 27 * U.CONVS[k][0] * U.CONVS[k][1])) for k in range(10)]
    idx += [int(offs[k] + 27 * U.CONVS[k][0] * U.CONVS[k][1] + 1) for k in (0, 5, 9)]  # biases
    idx += [len(p) - 5, len(p) - 1]  # head
    ok = 0
    for i in idx:
        e = 1e-6 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += e
        pm[i] -= e
        fd = (U.loss_grad(pp, delta, target, -0.7, 0.3, 0.8)[0] - U.loss_grad(pm, delta, target, -0.7, 0.3, 0.8)[0]) / (2 * e)
        ok += abs(fd - g[i]) <= 1e-5 * max(abs(fd), 1e-3)
    assert ok >= len(idx) - 1  # a ReLU kink may sit inside one stencil of the difference


def test_target_is_delta_in_the_linear_limit():
    """With kappa = 0 the solution satisfies nu L chi = src delta (+ const), so T = delta."""
    from paper_2604_15434_gb300 import synth

    n = 16
    d = synth.lognormal_delta(n, -2.0, 1.0, 5)
    c = O.coefficients(-0.2, -0.4, 1.0)  # C4 = 0: no screening
    assert c["kappa"] == 0.0
    chi, info, st = O.scalar_solve(d, -0.2, -0.4, 1.0, 1e-13)
    L = O.apply_N(chi, 1.0, 0.0)
    T = c["nu"] * L / c["src"]
    assert np.abs((T - T.mean()) - (d - d.mean())).max() < 1e-9
