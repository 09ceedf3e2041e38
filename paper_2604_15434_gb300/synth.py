"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and the oracle tests.

This module holds none of the method's arithmetic.  It only draws Gaussian random
fields with a power-law spectrum and displaces particles from a lattice, the
stand-ins for the paper's CAMB + MPGRAFIC 2LPT initial conditions (Sec. 3.6.2),
which are not available here.  Everything is generated on the host in float64 with
``numpy.random.default_rng(seed)`` so both sides of a comparison see the same bytes.

Box units throughout: the box is [0, 1)^3, a mesh of n cells has cell size 1/n and
cell centres at (i + 1/2)/n, arrays are indexed [z, y, x] (x fastest in memory), and
particle coordinates are stored as a [3, N] array of rows (x, y, z).
"""
from __future__ import annotations

import numpy as np

try:  # multithreaded FFTs when scipy is present (it is on every supported machine)
    import scipy.fft as _fft

    def _rfftn(a):
        return _fft.rfftn(a, workers=-1)

    def _irfftn(a, s):
        return _fft.irfftn(a, s=s, axes=(0, 1, 2), workers=-1)
except ImportError:  # pragma: no cover
    def _rfftn(a):
        return np.fft.rfftn(a)

    def _irfftn(a, s):
        return np.fft.irfftn(a, s=s, axes=(0, 1, 2))


def _wavenumbers(n):
    m = np.fft.fftfreq(n) * n
    mr = np.fft.rfftfreq(n) * n
    return m[:, None, None], m[None, :, None], mr[None, None, :]


def gaussian_field(n: int, slope: float, sigma: float, seed: int, nyquist_cutoff: bool = False) -> np.ndarray:
    """Zero-mean Gaussian field on n^3 cells with P(k) ~ k^slope (times exp(-(k/k_Nyq)^2) if asked).

    White noise is drawn in real space, filtered by sqrt(P) in Fourier space, and the
    result is rescaled to standard deviation ``sigma``.  k/k_Nyq = 2|m|/n for integer
    wavenumber m, so the box size only sets units and drops out.
    """
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((n, n, n))
    kz, ky, kx = _wavenumbers(n)
    m2 = kz * kz + ky * ky + kx * kx
    amp = np.zeros(m2.shape)
    nz = m2 > 0
    amp[nz] = m2[nz] ** (slope / 4.0)
    if nyquist_cutoff:
        amp *= np.exp(-0.5 * m2 * (2.0 / n) ** 2)
    g = _irfftn(_rfftn(w) * amp, (n, n, n))
    g -= g.mean()
    return g * (sigma / g.std())


def zeldovich_particles(n_side: int, slope: float, sigma: float, seed: int,
                        nyquist_cutoff: bool = False) -> np.ndarray:
    """n_side^3 particles at cell centres displaced by the Zel'dovich field of a Gaussian delta.

    x = q + Psi(q) with div Psi = -delta_lin, i.e. Psi_k = i k delta_k / k^2.
    Returns positions [3, n_side^3] wrapped into [0, 1).
    """
    n = n_side
    d = gaussian_field(n, slope, sigma, seed, nyquist_cutoff)
    dk = _rfftn(d)
    kz, ky, kx = _wavenumbers(n)
    k2 = (2.0 * np.pi) ** 2 * (kz * kz + ky * ky + kx * kx)
    k2[0, 0, 0] = 1.0
    q = (np.arange(n) + 0.5) / n
    pos = np.empty((3, n ** 3))
    for row, kk in ((0, kx), (1, ky), (2, kz)):
        disp = _irfftn(1j * (2.0 * np.pi * kk) * dk / k2, (n, n, n))
        if row == 0:
            base = np.broadcast_to(q[None, None, :], (n, n, n))
        elif row == 1:
            base = np.broadcast_to(q[None, :, None], (n, n, n))
        else:
            base = np.broadcast_to(q[:, None, None], (n, n, n))
        x = (base + disp).ravel()
        x = x - np.floor(x)
        x[x >= 1.0] = 0.0
        pos[row] = x
    return pos


def lognormal_delta(n: int, slope: float, sigma_ln: float, seed: int) -> np.ndarray:
    """delta = exp(g)/<exp(g)> - 1 for a Gaussian g with P(k) ~ k^slope and std(g) = sigma_ln."""
    g = gaussian_field(n, slope, sigma_ln, seed)
    rho = np.exp(g)
    return rho / rho.mean() - 1.0


def velocities_zero(npart: int) -> np.ndarray:
    return np.zeros((3, npart))


def sample_box_params(count: int, seed: int, accept=None):
    """Draw (alpha_B0, alpha_M0, a) with alpha_B0 ~ U[-2, 0], alpha_M0 ~ U[0, 1], a ~ U[0.3, 1].

    ``accept(alpha_B0, alpha_M0, a) -> bool`` lets the caller reject a draw (for example a
    near-singular one); rejected draws are replaced from the same stream, in order.
    Returns a list of (alpha_B0, alpha_M0, a, n_rejected_before_this_one).
    """
    rng = np.random.default_rng(seed)
    out = []
    rej = 0
    while len(out) < count:
        aB = rng.uniform(-2.0, 0.0)
        aM = rng.uniform(0.0, 1.0)
        a = rng.uniform(0.3, 1.0)
        if accept is not None and not accept(aB, aM, a):
            rej += 1
            continue
        out.append((aB, aM, a, rej))
    return out


def sample_box_sizes(count: int, seed: int, choices=(64, 128, 256)):
    rng = np.random.default_rng(seed)
    return [int(choices[i]) for i in rng.integers(0, len(choices), size=count)]
