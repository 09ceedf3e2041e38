"""The seeded synthetic inputs (the workload recipe both sides of every comparison use):
moments, spectral slope, seeding, the Zel'dovich displacement and the box samplers."""
import numpy as np
import pytest

import oracle as O
from paper_2604_15434_gb300 import synth


def _shell_power(g):
    n = g.shape[0]
    p = np.abs(np.fft.rfftn(g)) ** 2
    m = np.fft.fftfreq(n) * n
    mr = np.fft.rfftfreq(n) * n
    k = np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + mr[None, None, :] ** 2)
    ks, ps = [], []
    for lo in range(2, n // 4):
        sel = (k >= lo) & (k < lo + 1)
        ks.append(k[sel].mean())
        ps.append(p[sel].mean())
    return np.log(ks), np.log(ps)


@pytest.mark.parametrize("slope", [-2.0, -1.5])
def test_gaussian_field_moments_slope_and_seeding(slope):
    g = synth.gaussian_field(64, slope, 1.5, 7)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.5) < 1e-12
    lk, lp = _shell_power(g)
    fit = np.polyfit(lk, lp, 1)[0]
    assert abs(fit - slope) < 0.25, fit
    assert np.array_equal(g, synth.gaussian_field(64, slope, 1.5, 7))
    assert not np.array_equal(g, synth.gaussian_field(64, slope, 1.5, 8))


def test_nyquist_cutoff_removes_small_scale_power():
    a = synth.gaussian_field(32, -1.5, 1.0, 3)
    b = synth.gaussian_field(32, -1.5, 1.0, 3, nyquist_cutoff=True)
    pa, pb = np.abs(np.fft.rfftn(a)) ** 2, np.abs(np.fft.rfftn(b)) ** 2
    hi = (slice(12, 20), slice(12, 20), slice(12, 17))  # |m| near the Nyquist frequency
    assert pb[hi].sum() / pb.sum() < 0.5 * pa[hi].sum() / pa.sum()


def test_lognormal_delta_mean_floor_and_log_width():
    d = synth.lognormal_delta(48, -2.0, 1.5, 1003)
    assert abs(d.mean()) < 1e-12 and d.min() > -1.0
    assert abs(np.log1p(d).std() - 1.5) < 1e-9  # log(1 + delta) = g - log <exp g>


def _lowpass(f, mmax):
    n = f.shape[0]
    F = np.fft.rfftn(f)
    m = np.fft.fftfreq(n) * n
    mr = np.fft.rfftfreq(n) * n
    k = np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + mr[None, None, :] ** 2)
    F[k > mmax] = 0
    return np.fft.irfftn(F, s=f.shape, axes=(0, 1, 2))


def test_zeldovich_particles_follow_the_linear_density():
    """Positions lie in [0, 1) and, at small amplitude, the CIC density of the displaced
    lattice is the linear field on large scales (div Psi = -delta_lin; the CIC window only
    damps the modes near the Nyquist frequency)."""
    n = 32
    pos = synth.zeldovich_particles(n, -1.5, 0.05, 11, nyquist_cutoff=True)
    assert pos.shape == (3, n ** 3) and pos.min() >= 0.0 and pos.max() < 1.0
    d = O.density(O.deposit_cic(pos, n), pos.shape[1])
    lin = synth.gaussian_field(n, -1.5, 0.05, 11, nyquist_cutoff=True)
    a, b = _lowpass(d, n // 8), _lowpass(lin, n // 8)
    assert np.corrcoef(a.ravel(), b.ravel())[0, 1] > 0.98
    assert 0.95 < a.std() / b.std() < 1.0


def test_box_samplers_ranges_and_rejection_bookkeeping():
    draws = synth.sample_box_params(200, 5)
    a = np.array([x[:3] for x in draws])
    assert (a[:, 0] >= -2).all() and (a[:, 0] <= 0).all() and (a[:, 1] >= 0).all() and (a[:, 1] <= 1).all()
    assert (a[:, 2] >= 0.3).all() and (a[:, 2] <= 1).all() and all(x[3] == 0 for x in draws)
    kept = synth.sample_box_params(20, 5, accept=lambda b, m, s: b > -1.0)
    assert all(x[0] > -1.0 for x in kept) and kept[-1][3] > 0
    assert [x[:3] for x in kept][:1] == [x[:3] for x in draws if x[0] > -1.0][:1]
    sizes = synth.sample_box_sizes(50, 9)
    assert set(sizes) <= {64, 128, 256} and sizes == synth.sample_box_sizes(50, 9)
